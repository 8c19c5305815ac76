"""Batched ensembles of independent grids of uneven size.

All members advance inside one CUDA graph: the capture forks the members over
several streams (independent branches of the graph) and joins them, so one
graph launch advances every member by n steps with the members' kernels free
to overlap on the GPU.  The same members can be stepped one by one for
comparison.  Members never exchange data.
"""
import numpy as np
import torch

from .workload import body_tensor, grid_from_workload


class Member:
    def __init__(self, wl, precision):
        self.wl = wl
        self.grid = grid_from_workload(wl, precision)
        self.u = [torch.tensor(np.asarray(a), dtype=self.grid.dtype, device="cuda").contiguous() for a in wl.u0]
        self.body = body_tensor(wl)
        self.dt = wl.dt

    def cells(self):
        return int(np.prod(self.wl.n))

    def step(self, n):
        self.grid.step(self.u, self.dt, n, body=self.body)


class Ensemble:
    def __init__(self, workloads, precision="mixed", streams=32, tune=False):
        self.members = [Member(wl, precision) for wl in workloads]
        self.nstreams = max(1, int(streams))
        self.graph = None
        self.graph_steps = 0
        if tune:
            from . import autotune
            for m in self.members:
                autotune.tune(m.grid, m.u, m.dt, m.body)

    def cells(self):
        return sum(m.cells() for m in self.members)

    def snapshot(self):
        return [([x.clone() for x in m.u], m.body.clone() if m.body is not None else None) for m in self.members]

    def restore(self, snap):
        for m, (u, b) in zip(self.members, snap):
            for x, y in zip(m.u, u):
                x.copy_(y)
            if b is not None:
                m.body.copy_(b)

    def step_sequential(self, n):
        """Every member advanced by n steps, launched member after member on the current stream."""
        cur = torch.cuda.current_stream()
        for m in self.members:
            m.grid.set_stream(cur)
            m.step(n)

    def capture(self, n):
        """Record n steps of every member into one CUDA graph (members on parallel branches)."""
        main = torch.cuda.Stream()
        branches = [torch.cuda.Stream() for _ in range(self.nstreams)]
        # warm-up on the capture streams (kernel attributes, lazily created state)
        for i, m in enumerate(self.members):
            m.grid.set_stream(branches[i % self.nstreams])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=main):
            fork = torch.cuda.Event()
            fork.record(main)
            for s in branches:
                s.wait_event(fork)
            for i, m in enumerate(self.members):
                m.grid.set_stream(branches[i % self.nstreams])
                m.step(n)
            for s in branches:
                main.wait_stream(s)
        self.graph, self.graph_steps = g, n
        return g

    def replay(self):
        self.graph.replay()
