"""Batched ensembles of independent grids of uneven size.

All members advance inside one CUDA graph: the capture forks the members over
several streams (independent branches of the graph) and joins them, so one
graph launch advances every member by n steps with the members' kernels free
to overlap on the GPU.  The same members can be stepped one by one for
comparison.  Members never exchange data.

Forward + adjoint (the gradient of a loss of every member's final state,
§2.4.1) runs as windows of steps: a forward graph advances all members by one
window (a flat checkpoint copy of every member's state before each), and a
window graph re-runs one window from its checkpoint keeping each step's state,
then takes that window's adjoint steps (fs_step_adjoint with the force
sensitivity in device memory, so the graph holds no host copy) in reverse.
Graphs have fixed buffer addresses, so one window graph serves every window:
the checkpoint is copied into its start buffer before each launch.
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
        # warm-up: one step of every member on its capture stream (kernel attributes, lazily
        # created state), then the states restored
        snap = self.snapshot()
        for i, m in enumerate(self.members):
            st = branches[i % self.nstreams]
            m.grid.set_stream(st)
            with torch.cuda.stream(st):
                m.step(1)
        torch.cuda.synchronize()
        self.restore(snap)
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

    # ---- forward + adjoint -------------------------------------------------------------------
    def _flat_state(self):
        """One flat device buffer holding every member's fields and body state (views per member)."""
        sizes = []
        for m in self.members:
            sizes += [x.numel() * x.element_size() for x in m.u]
            sizes.append(m.body.numel() * 8 if m.body is not None else 0)
        total = sum((b + 255) // 256 * 256 for b in sizes)
        buf = torch.empty(total, dtype=torch.uint8, device="cuda")
        views, off, i = [], 0, 0
        for m in self.members:
            us = []
            for x in m.u:
                n = x.numel() * x.element_size()
                us.append(buf[off:off + n].view(x.dtype).view(x.shape))
                off += (n + 255) // 256 * 256
                i += 1
            b = None
            if m.body is not None:
                b = buf[off:off + 32].view(torch.float64)
                off += 256
            views.append((us, b))
        return buf, views

    def setup_adjoint(self, window, windows, weights):
        """Buffers of the windowed forward + adjoint sweep: `windows` checkpoints of every member's state
        (one flat buffer each), the window-start state, `window` per-step tapes, the adjoints, and the
        loss weights (per member, per component: dJ/du_T = weights * u_T, the gradient of
        1/2 sum weights u_T^2)."""
        self.window, self.windows = int(window), int(windows)
        self.work, self.work_v = self._flat_state()
        self.start, self.start_v = self._flat_state()
        self.chk = [self._flat_state() for _ in range(self.windows)]
        self.tape = [self._flat_state() for _ in range(self.window)]
        self.lam, self.lam_v = self._flat_state()
        self.weights = weights
        self.zero_dJdF = torch.zeros(2, dtype=torch.float64, device="cuda")
        # warm-up (lazily allocated adjoint buffers, kernel attributes) before any capture
        cur = torch.cuda.current_stream()
        for m, (u, b) in zip(self.members, self.work_v):
            m.grid.set_stream(cur)
            for x, y in zip(u, m.u):
                x.copy_(y)
            if b is not None:
                b.copy_(m.body)
        self.lam.zero_()
        for m, (u, b), (lu, lb) in zip(self.members, self.work_v, self.lam_v):
            m.grid.step_adjoint(u, lu, m.dt, body_n=b, lam_body=lb, dJdF=self.zero_dJdF)
        torch.cuda.synchronize()

    def _member_window(self, i, forward_only):
        m = self.members[i]
        su, sb = self.start_v[i] if not forward_only else self.work_v[i]
        wu, wb = self.work_v[i]
        lu, lb = self.lam_v[i]
        if not forward_only:
            for x, y in zip(wu, su):
                x.copy_(y)
            if wb is not None:
                wb.copy_(sb)
        if forward_only:
            m.grid.step(wu, m.dt, self.window, body=wb)
            return
        for t in range(self.window):
            tu, tb = self.tape[t][1][i]
            for x, y in zip(tu, wu):
                x.copy_(y)
            if tb is not None:
                tb.copy_(wb)
            m.grid.step(wu, m.dt, 1, body=wb)
        for t in range(self.window - 1, -1, -1):
            tu, tb = self.tape[t][1][i]
            m.grid.step_adjoint(tu, lu, m.dt, body_n=tb, lam_body=lb, dJdF=self.zero_dJdF)

    def capture_windows(self, streams=None):
        """Two CUDA graphs over all members on parallel branches: `fwd` advances every member by one
        window of steps (in place), `win` re-runs one window from the window-start state keeping each
        step's state and then takes the window's adjoint steps in reverse."""
        nst = self.nstreams if streams is None else streams
        main = torch.cuda.Stream()
        branches = [torch.cuda.Stream() for _ in range(nst)]
        graphs = []
        for fwd in (True, False):
            g = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=main):
                fork = torch.cuda.Event()
                fork.record(main)
                for s in branches:
                    s.wait_event(fork)
                for i, m in enumerate(self.members):
                    st = branches[i % nst]
                    m.grid.set_stream(st)
                    with torch.cuda.stream(st):
                        self._member_window(i, fwd)
                for s in branches:
                    main.wait_stream(s)
            graphs.append(g)
        self.g_fwd, self.g_win = graphs
        cur = torch.cuda.current_stream()
        for m in self.members:
            m.grid.set_stream(cur)

    def load_initial(self):
        for m, (u, b) in zip(self.members, self.work_v):
            for x, y in zip(u, m.u):
                x.copy_(y)
            if b is not None:
                b.copy_(m.body)

    def _seed_loss(self):
        for (u, _), (lu, lb), w in zip(self.work_v, self.lam_v, self.weights):
            for x, y, v in zip(lu, u, w):
                x.copy_(y * v)
            if lb is not None:
                lb.zero_()

    def fwd_adj_graph(self):
        """Forward over windows * window steps keeping a checkpoint per window, then the reverse
        sweep window by window (each window's forward recomputed from its checkpoint): 2 * windows
        graph launches and one flat copy per window.  Leaves dJ/du_0 in lam_v."""
        self.load_initial()
        for j in range(self.windows):
            self.chk[j][0].copy_(self.work)
            self.g_fwd.replay()
        self._seed_loss()
        for j in range(self.windows - 1, -1, -1):
            self.start.copy_(self.chk[j][0])
            self.g_win.replay()

    def fwd_adj_sequential(self):
        """The same sweep launched member after member (no graph): each member's forward over all
        windows with its checkpoints, then its reverse sweep."""
        cur = torch.cuda.current_stream()
        self.load_initial()
        for m in self.members:
            m.grid.set_stream(cur)
        for i in range(len(self.members)):
            wu, wb = self.work_v[i]
            for j in range(self.windows):
                cu, cb = self.chk[j][1][i]
                for x, y in zip(cu, wu):
                    x.copy_(y)
                if cb is not None:
                    cb.copy_(wb)
                self._member_window(i, True)
            lu, lb = self.lam_v[i]
            for x, y, v in zip(lu, wu, self.weights[i]):
                x.copy_(y * v)
            if lb is not None:
                lb.zero_()
            su, sb = self.start_v[i]
            for j in range(self.windows - 1, -1, -1):
                cu, cb = self.chk[j][1][i]
                for x, y in zip(su, cu):
                    x.copy_(y)
                if sb is not None:
                    sb.copy_(cb)
                self._member_window(i, False)
