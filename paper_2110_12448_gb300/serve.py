"""Continuous-batching request loop for solidification runs.

Requests (a seeded workload, a step count, a precision) arrive over time.
The loop admits a request as soon as its device memory fits the HBM budget
(a fraction of the GPU's memory) and a group slot is free, keeps every
admitted run's fields resident, and advances all running runs together with
one persistent launch per (dimension, scheme, precision) class per step
(``pf_group_step``, replayed from a CUDA graph).  Between chunks of steps it
retires finished runs (observation + fields copied to the host), frees their
memory and admits waiting ones.  A chunk never takes a run past its own step
count, so every run advances by exactly its requested number of steps with
the same per-cell arithmetic as when it runs alone: results are identical
alone and in the mix.

``Scheduler`` holds the admission policy and bookkeeping and touches no
device; ``Server`` drives the C-ABI through the binding.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    workload: object            # synth.Workload
    steps: int
    precision: str = "f32"
    arrival_s: float = 0.0       # offset from the start of the run
    keep_fields: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    arrival_s: float
    admit_s: float
    done_s: float
    steps: int
    cells: int
    obs: dict
    fields: Optional[tuple] = None

    @property
    def time_to_result(self) -> float:
        return self.done_s - self.arrival_s


class Scheduler:
    """Admission by memory budget and slot count; FIFO with backfill.

    bytes_of(request) gives the device bytes a request needs while it runs.
    The head of the queue is admitted first; with backfill, later requests
    that fit are admitted while the head waits (the head is never starved:
    once it has waited `max_bypass` admissions, nothing else jumps it)."""

    def __init__(self, budget_bytes: int, max_running: int, bytes_of: Callable[[Request], int],
                 backfill: bool = True, max_bypass: int = 8):
        self.budget = int(budget_bytes)
        self.max_running = int(max_running)
        self.bytes_of = bytes_of
        self.backfill = backfill
        self.max_bypass = max_bypass
        self.queue: List[Request] = []
        self.running: Dict[int, Request] = {}
        self.used = 0
        self._bypassed = 0

    def submit(self, r: Request):
        need = self.bytes_of(r)
        if need > self.budget:
            raise ValueError(f"request {r.rid} needs {need} bytes, above the whole budget {self.budget}")
        self.queue.append(r)

    def admissible(self) -> List[Request]:
        """Requests to admit now (removed from the queue, counted as running)."""
        out = []
        i = 0
        while i < len(self.queue) and len(self.running) < self.max_running:
            r = self.queue[i]
            if i > 0 and self._bypassed >= self.max_bypass:
                break  # the waiting head has been jumped often enough
            need = self.bytes_of(r)
            if self.used + need <= self.budget:
                self.queue.pop(i)
                self.running[r.rid] = r
                self.used += need
                out.append(r)
                self._bypassed = self._bypassed + 1 if i > 0 else 0
                continue
            if not self.backfill:
                break
            i += 1
        return out

    def retire(self, rid: int):
        r = self.running.pop(rid)
        self.used -= self.bytes_of(r)

    @property
    def idle(self) -> bool:
        return not self.queue and not self.running


def percentile(xs, q):
    if not xs:
        return float("nan")
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


class Server:
    """Drives the batched C-ABI path for a stream of requests.  The running
    requests are spread over `n_streams` groups, each on its own CUDA stream
    (a request joins the group with the fewest cells), so that one group's
    launches overlap another's: the 2D and 3D classes, and the tails of each
    group's persistent launches."""

    def __init__(self, budget_frac: float = 0.8, max_running: int = 256, chunk: int = 100, use_graph: bool = True,
                 device: int = 0, budget_bytes: Optional[int] = None, n_streams: int = 2):
        import torch

        from . import native as N
        self.N = N
        self.torch = torch
        torch.cuda.set_device(device)
        total = torch.cuda.mem_get_info()[1]
        self.budget = int(budget_bytes if budget_bytes is not None else budget_frac * total)
        self.streams = [torch.cuda.Stream() for _ in range(max(1, int(n_streams)))]
        self.stream = self.streams[0]
        self.chunk = int(chunk)
        self.use_graph = use_graph
        self.max_running = max_running
        self.sched = Scheduler(self.budget, max_running, self._bytes_of)
        self._work_cap = 1 << 20  # 32 MB of work items
        self.groups = [N.Group(max_running, self._work_cap, stream=st) for st in self.streams]
        self.load = [0] * len(self.groups)  # cells running in each group
        self.where: Dict[int, int] = {}
        self.sims: Dict[int, object] = {}
        self.target: Dict[int, int] = {}
        self.admit_t: Dict[int, float] = {}
        self.results: List[Result] = []
        self.cell_steps = 0
        self.cell_steps_by_dim = {2: 0, 3: 0}
        self.max_running_seen = 0
        self.peak_bytes = 0

    def _params(self, r: Request):
        w = r.workload
        return self.N.make_params(w.dim, w.nx, w.ny, w.nz, w.h, w.dt, w.k, w.eps4, w.lam, w.D, w.U0, w.scheme,
                                  r.precision, max_grains=max(1, w.n_grains), max_seeds=max(1, len(w.seeds)))

    def _bytes_of(self, r: Request) -> int:
        n = self.N.required_bytes(self._params(r))
        if n == 0:
            raise ValueError(f"request {r.rid}: invalid parameters")
        return n

    def _admit(self, r: Request, now: float):
        k = min(range(len(self.groups)), key=lambda i: self.load[i])
        with self.torch.cuda.stream(self.streams[k]):
            s = self.N.Sim.from_workload(r.workload, r.precision, stream=self.streams[k])
        self.groups[k].add(s)
        self.where[r.rid] = k
        self.load[k] += s.n_cells
        self.sims[r.rid] = s
        self.target[r.rid] = r.steps
        self.admit_t[r.rid] = now

    def _retire(self, rid: int, now_fn):
        s = self.sims.pop(rid)
        r = self.sched.running[rid]
        k = self.where.pop(rid)
        self.groups[k].remove(s)
        self.load[k] -= s.n_cells
        obs = s.observe(-1, allow_nonfinite=True)
        fields = s.get_fields() if r.keep_fields else None
        self.results.append(Result(rid, r.arrival_s * self._scale, self.admit_t.pop(rid), now_fn(), r.steps, s.n_cells,
                                   obs, fields))
        self.target.pop(rid)
        s.close()
        self.sched.retire(rid)

    def run(self, requests: List[Request], time_scale: float = 1.0) -> List[Result]:
        """Serve `requests` (arrival offsets in seconds, scaled by time_scale)
        in wall-clock time; returns the results in completion order."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        self._scale = time_scale
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        k = 0
        while k < len(pending) or not self.sched.idle:
            t = now()
            while k < len(pending) and pending[k].arrival_s * time_scale <= t:
                self.sched.submit(pending[k])
                k += 1
            for r in self.sched.admissible():
                self._admit(r, now())
            if not self.sims:
                if k < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[k].arrival_s * time_scale - now())))
                continue
            # a chunk never passes any running run's own step count
            n = min([self.chunk] + [self.target[rid] - self.sims[rid].steps_done for rid in self.sims])
            if n > 0:
                for g in self.groups:  # each on its own stream, queued back to back
                    if len(g.members):
                        g.step(n, use_graph=self.use_graph)
                self.cell_steps += n * sum(s.n_cells for s in self.sims.values())
                for s in self.sims.values():
                    self.cell_steps_by_dim[s.p.dim] += n * s.n_cells
                self.max_running_seen = max(self.max_running_seen, len(self.sims))
                self.peak_bytes = max(self.peak_bytes, self.sched.used)
            for st in self.streams:  # bound the queue depth: times below are device-complete
                st.synchronize()
            for rid in [rid for rid in self.sims if self.sims[rid].steps_done >= self.target[rid]]:
                self._retire(rid, now)
        self.wall_s = now()
        return self.results

    def summary(self) -> dict:
        ttr = [r.time_to_result for r in self.results]
        return {"requests": len(self.results), "p50_s": percentile(ttr, 50), "p99_s": percentile(ttr, 99),
                "wall_s": self.wall_s, "glups": self.cell_steps / self.wall_s / 1e9 if self.wall_s > 0 else 0.0,
                "cell_updates_2d": self.cell_steps_by_dim[2], "cell_updates_3d": self.cell_steps_by_dim[3],
                "max_running": self.max_running_seen, "peak_bytes": self.peak_bytes, "budget_bytes": self.budget}

    def close(self):
        for rid in list(self.sims):
            s = self.sims.pop(rid)
            self.groups[self.where.pop(rid)].remove(s)
            s.close()
        for g in self.groups:
            g.close()
