"""A batch of instances stepped as several groups, each on its own CUDA
stream.

One group advances all its members by one persistent launch per step.  Its
last wave of work items leaves SMs idle while the slowest warps finish, and
the next launch cannot start before that.  Two groups on two streams, each
with half of the instances, fill each other's tails: on GB300 the ten-instance
1024^2 sweep runs 7 % faster as two groups than as one (three or five groups
gain no more).  The instances are independent, so no group waits on another
within a step.

`Batch.step` forks from the caller's stream (every group stream waits on an
event recorded there) and joins back (the caller's stream waits on an event
of every group stream), so work queued on the caller's stream before and
after it is ordered as for a single launch.  Host orchestration only: the
steps are the library's group launches (pf_group_step), the reductions its
group observes (pf_group_observe).
"""
from __future__ import annotations

from . import native as N


class Batch:
    """`workloads` split round-robin over `n_streams` groups (fewer when there
    are fewer workloads), each group and its members on their own stream.
    `tile` as autotune.tune returns it: (block_x, block_y, sweep) for the
    members, and at depth 2 the group's temporal-blocking depth and band."""

    def __init__(self, workloads, precision="f32", n_streams=2, tile=None, device="cuda"):
        import torch
        if not workloads:
            raise ValueError("Batch: no workloads")
        n = max(1, min(int(n_streams), len(workloads)))
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n)]
        self.order = []   # (group index, member index) of each workload, in workload order
        self.parts = [[] for _ in range(n)]
        for i, w in enumerate(workloads):
            k = i % n
            self.order.append((k, len(self.parts[k])))
            self.parts[k].append(w)
        self.sims = []    # per group, its members
        self.groups = []
        from .autotune import split
        for st, part in zip(self.streams, self.parts):
            ss = [N.Sim.from_workload(w, precision, stream=st) for w in part]
            if tile:
                for s in ss:
                    s.set_tile(*split(tile)[0])
            g = N.Group(len(ss), sum(N.Group.work_items(s) for s in ss), stream=st, device=device)
            for s in ss:
                g.add(s)
            if tile:
                g.set_depth(*split(tile)[1])
            self.sims.append(ss)
            self.groups.append(g)

    @property
    def members(self):
        """the instances in workload order"""
        return [self.sims[k][j] for k, j in self.order]

    @property
    def n_cells(self) -> int:
        return sum(s.n_cells for ss in self.sims for s in ss)

    @property
    def steps_done(self) -> int:
        return self.sims[0][0].steps_done

    def step(self, n: int = 1, use_graph: bool = True, stream=None):
        """Advance every instance by n steps: fork from `stream` (default the
        current stream), each group's launches on its own stream, join back."""
        import torch
        main = stream if stream is not None else torch.cuda.current_stream()
        if len(self.groups) == 1 and self.streams[0] == main:
            self.groups[0].step(n, use_graph)
            return
        fork = torch.cuda.Event()
        fork.record(main)
        for st in self.streams:
            st.wait_event(fork)
        for g in self.groups:
            g.step(n, use_graph)
        for st in self.streams:
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)

    def observe(self, grain: int = -1, allow_nonfinite=False) -> list:
        """pf_group_observe of every group (one synchronisation each); dicts in
        workload order."""
        per = [g.observe(grain, allow_nonfinite) for g in self.groups]
        return [per[k][j] for k, j in self.order]

    def close(self):
        for g in self.groups:
            g.close()
        for ss in self.sims:
            for s in ss:
                s.close()
        self.groups, self.sims = [], []
