"""Tile autotuner for the fused step kernels.

For a batch of instances of one class (dimension, scheme, precision, grid
size) it times each candidate tile -- the sweep length in 2D; the block
shape and sweep length in 3D -- on synthetic seed states, in one persistent
launch per step exactly as the batched path runs, and keeps the fastest.
Wave quantisation (work items vs resident warps or blocks) is what the
choice mostly trades against the per-sweep prologue (about 2.5 rows of extra
work per work item), so the answer depends on the batch size as well as the
grid.  Besides a fixed list, the candidates include, for k = 1, 2, ... waves,
the shortest sweep whose work list fits in k waves of resident units
(``pf_resident_units``), which balances the persistent launch with the least
prologue for that wave count.

It also races the temporal-blocking depth (``pf_group_set_depth``): depth 2
advances two steps per wavefront over bands of sweeps, so that the
intermediate level is read back from L2.  A band must hold enough work items
to fill the GPU by itself (every band is one launch), so the depth-2
candidates are, for a few sweep lengths, the fewest sweeps per band that fill
one and two waves of resident units.  A tile is then (block_x, block_y, sweep)
at depth 1 and (block_x, block_y, sweep, 2, band_sweeps) at depth 2
(``split``).  Results are cached per device in ``_build/autotune.json``.
"""
from __future__ import annotations

import json
import os
import threading

CANDIDATES_2D = [(64, 1, s) for s in (12, 14, 16, 18, 20, 22, 24, 26, 28, 32, 36, 40, 48, 64, 96, 128)]
CANDIDATES_3D = [(34, by, s) for by in (18, 10) for s in (16, 32, 64)]

_HERE = os.path.dirname(os.path.abspath(__file__))
_CACHE = os.path.join(_HERE, "_build", "autotune.json")
_lock = threading.Lock()


def work_items(w, tile) -> int:
    """Work items of one instance for tile (block_x, block_y, sweep), the
    library's decomposition: 2D (block_x - 4)-column strips times sweep-row
    bands; 3D (block_x - 4) x (block_y - 4) columns times sweep-plane bands."""
    bx, by, sw = tile
    n = -(-w.nx // (bx - 4)) * -(-(w.ny if w.dim == 2 else w.nz) // sw)
    return n if w.dim == 2 else n * -(-w.ny // (by - 4))


def wave_aligned(workloads, bx, by, resident, max_waves=8, min_sweep=8):
    """For k = 1 .. max_waves: the shortest sweep whose work list over all
    `workloads` fits in k waves of `resident` units."""
    depth = max(w.ny if w.dim == 2 else w.nz for w in workloads)
    out = []
    for k in range(1, max_waves + 1):
        for sw in range(min_sweep, depth + 1):
            if sum(work_items(w, (bx, by, sw)) for w in workloads) <= k * resident:
                if (bx, by, sw) not in out:
                    out.append((bx, by, sw))
                break
    return out


def split(tile):
    """(block_x, block_y, sweep) of the members and (depth, band_sweeps) of
    the group for a tile the tuner returned."""
    t = tuple(int(x) for x in tile)
    return t[:3], ((t[3], t[4]) if len(t) > 3 else (1, 1))


def bands(workloads, tile) -> int:
    """Bands of a depth-2 wavefront over `workloads` (the deepest instance's
    sweeps over the band height); 1 at depth 1."""
    (bx, by, sw), (depth, bs) = split(tile)
    if depth == 1:
        return 1
    return max(-(-(-(-(w.ny if w.dim == 2 else w.nz) // sw)) // bs) for w in workloads)


def depth_race(times) -> dict:
    """The fastest depth-1 and depth-2 candidates of a tuner's times."""
    out = {}
    for k, t in times.items():
        tile = tuple(int(x) for x in k.strip("()").split(","))
        d = split(tile)[1][0]
        if f"depth{d}_ms" not in out or t * 1e3 < out[f"depth{d}_ms"]:
            out[f"depth{d}_ms"], out[f"depth{d}_tile"] = t * 1e3, list(tile)
    return out


def wavefront_ok(w) -> bool:
    """Whether a workload can step as depth-2 wavefronts: not with a frozen
    temperature (one step clock per launch) or the two-kernel form."""
    return not getattr(w, "thermal", 0) and not getattr(w, "kernels", 0)


def band_candidates(workloads, tile, resident, waves=(1, 2)):
    """Depth-2 candidates for a depth-1 tile: for each wave count k, the
    fewest sweeps per band whose work items fill k waves of `resident` units,
    at most half the deepest instance's sweeps: a single band would be two
    whole-grid launches, the schedule of depth 1 (a batch too small to fill
    the GPU with one band gets two bands)."""
    bx, by, sw = tile
    per_band_row = sum(work_items(w, (bx, by, 1 << 30)) for w in workloads)  # items of one sweep row
    sweeps = max(-(-(w.ny if w.dim == 2 else w.nz) // sw) for w in workloads)
    out = []
    if sweeps < 2:
        return out
    for k in waves:
        bs = min(max(1, -(-k * resident // per_band_row)), -(-sweeps // 2))
        if (bx, by, sw, 2, bs) not in out:
            out.append((bx, by, sw, 2, bs))
    return out


def _key(device_name, w, precision, count, n_streams=1):
    ds = "|ds" if getattr(w, "thermal", 0) or getattr(w, "bc_x", 0) else ""  # the directional kernel variant
    ds += "|t0" if getattr(w, "time_level", 0) else ""
    ds += "|two" if getattr(w, "kernels", 0) else ""
    ds += f"|s{n_streams}" if n_streams > 1 else ""
    ds += "|d12"  # depths 1 and 2 raced
    return f"{device_name}|{w.dim}|{w.scheme}|{precision}|{w.nx}x{w.ny}x{w.nz}|n{count}{ds}"


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def tune(workloads, precision="f32", steps=24, repeats=2, use_cache=True, verbose=False, n_streams=1):
    """Best tile for a batch shaped like `workloads` (all of one class):
    (block_x, block_y, sweep), or (block_x, block_y, sweep, 2, band_sweeps)
    when depth-2 wavefronts win, timed under the schedule it will run with:
    the batch as `n_streams` groups on their own streams (batch.Batch), one
    group when 1.  Returns (tile, {tile: seconds per step})."""
    import torch

    from . import native as N
    w0 = workloads[0]
    n_streams = max(1, min(int(n_streams), len(workloads)))
    dev = torch.cuda.get_device_name()
    key = _key(dev, w0, precision, len(workloads), n_streams)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"]), cache[key]["times"]
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    # members of part k run on stream k (round-robin, as batch.Batch splits)
    part_of = [i % n_streams for i in range(len(workloads))]
    sims = [N.Sim.from_workload(w, precision, stream=streams[k]) for w, k in zip(workloads, part_of)]
    cands = list(CANDIDATES_2D if w0.dim == 2 else CANDIDATES_3D)
    resident = {}
    for bx, by in sorted({(t[0], t[1]) for t in cands}):
        try:
            for s in sims:
                s.set_tile(bx, by, 0)
            resident[(bx, by)] = sims[0].resident_units()
        except N.PfError:
            continue
        cands += [t for t in wave_aligned(workloads, bx, by, resident[(bx, by)]) if t not in cands]
    times = {}

    def race(tile):
        t3, (depth, bands) = split(tile)
        try:
            for s in sims:
                s.set_tile(*t3)
        except N.PfError:
            return
        groups = []
        for k, st in enumerate(streams):
            mine = [s for s, p in zip(sims, part_of) if p == k]
            g = N.Group(len(mine), sum(N.Group.work_items(s) for s in mine), stream=st)
            for s in mine:
                g.add(s)
            g.set_depth(depth, bands)
            g.step(4, use_graph=False)
            groups.append(g)
        main = torch.cuda.current_stream()
        best = float("inf")
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(main)
            for st in streams:
                st.wait_event(a)
            for g in groups:
                g.step(steps, use_graph=True)
            for st in streams:
                j = torch.cuda.Event()
                j.record(st)
                main.wait_event(j)
            b.record(main)
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3 / steps)
        for g in groups:
            g.close()
        times[str(tuple(tile))] = best
        if verbose:
            print(f"autotune {key} {tile}: {best * 1e3:.3f} ms/step", flush=True)

    for tile in cands:
        race(tile)
    # depth 2 on the best depth-1 tile of each block shape and on its shortest sweep
    if all(wavefront_ok(w) for w in workloads) and times:
        done1 = [(t, tuple(int(x) for x in k.strip("()").split(","))) for k, t in times.items()]
        for (bx, by), res in sorted(resident.items()):
            mine = sorted((t, c) for t, c in done1 if c[:2] == (bx, by))
            if not mine:
                continue
            for base in dict.fromkeys([mine[0][1], (bx, by, 8)]):
                # the groups' band launches run side by side: together they fill the waves
                for tile in band_candidates(workloads, base, res):
                    race(tile)
    for s in sims:
        s.close()
    tile = min(((t, tuple(int(x) for x in k.strip("()").split(","))) for k, t in times.items()))[1]
    with _lock:
        cache = _load()
        cache[key] = {"tile": list(tile), "times": times}
        _store(cache)
    return tile, times
