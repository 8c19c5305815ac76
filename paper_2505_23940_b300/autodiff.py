"""Differentiable rollouts: binomial ("revolve") checkpointing of time steps around
fs_step / fs_step_adjoint, and a torch.autograd.Function over a whole rollout.

The paper differentiates long rollouts with reverse-mode AD plus gradient
checkpointing (§2.4.1) and nested scans (§2.4.2).  Here the forward steps and
their hand-written adjoints are CUDA kernels; this module only decides which
states to keep, which segments to recompute, and in which order to call the
adjoint step.  State snapshots live in HBM as device tensors.

Schedule.  With s snapshot slots and t recomputation sweeps, at most
beta(s, t) = C(s + t, s) steps can be reversed (Griewank, "Achieving
logarithmic growth of temporal and spatial complexity in reverse automatic
differentiation", 1992).  To reverse steps [a, b) from a stored state at a with
s free slots, the schedule advances to a + d with d = beta(s, t - 1) for the
smallest t with beta(s, t) >= b - a, stores that state, reverses [a + d, b)
with s - 1 slots, releases the slot and reverses [a, a + d) with s slots.
"""
from math import comb

import torch

from . import fsstep as F


def _beta(s, t):
    return comb(s + t, s)


def revolve_schedule(n, slots):
    """Actions reversing n steps with `slots` snapshot slots (state 0 is always kept).

    Returns a list of tuples:
      ("advance", a, b)   run forward steps a .. b-1 from the working state at a
      ("store", slot, a)  copy the working state (at step a) into slot
      ("load", slot, a)   copy slot (holding the state at step a) into the working state
      ("adjoint", a)      working state is the state at step a: run the adjoint of step a
    Slot 0 holds the initial state.
    """
    ops = []
    # the recursion rev(a, b, free, base) of the binomial schedule, run from an explicit stack (a
    # schedule with a slot per step nests n levels deep); `free` is always a suffix of the slot list
    # 1 .. slots - 1, held as its first index k (free slots k + 1 .. slots - 1)
    nfree0 = slots - 1
    stack = [(0, n, 0, 0)]
    while stack:
        a, b, k, base_slot = stack.pop()
        # the state at a is held in base_slot
        n_ = b - a
        if n_ <= 0:
            continue
        if n_ == 1:
            ops.append(("load", base_slot, a))
            ops.append(("adjoint", a))
            continue
        s = nfree0 - k
        if s <= 0:
            for t in range(b - 1, a - 1, -1):
                ops.append(("load", base_slot, a))
                if t > a:
                    ops.append(("advance", a, t))
                ops.append(("adjoint", t))
            continue
        t = 1
        while _beta(s, t) < n_:
            t += 1
        d = max(1, min(n_ - 1, _beta(s, t - 1)))
        m = a + d
        ops.append(("load", base_slot, a))
        ops.append(("advance", a, m))
        slot = k + 1
        ops.append(("store", slot, m))
        stack.append((a, m, k, base_slot))       # second: the first part, with the same slots
        stack.append((m, b, k + 1, slot))        # first: the rest, from the stored state
    return ops


def split_schedule(n, slots):
    """(stores, rest): the forward prefix of the schedule (everything before its first
    adjoint) as {step: slot} for the states it stores, and the remaining actions.  A
    forward pass that keeps those states and the state at step n - 1 (the working state
    of the first remaining action, the adjoint of step n - 1) needs no recomputation
    until the schedule's first reload."""
    ops = revolve_schedule(n, slots)
    i = next(k for k, op in enumerate(ops) if op[0] == "adjoint")
    stores = {op[2]: op[1] for op in ops[:i] if op[0] == "store"}
    return stores, ops[i:]


def simulate(n, slots):
    """Replay a schedule on integers: returns (adjoint step order, forward steps recomputed)."""
    work, mem, order, fwd = None, {}, [], 0
    mem[0] = 0
    for op in revolve_schedule(n, slots):
        if op[0] == "load":
            assert mem.get(op[1]) == op[2], op
            work = op[2]
        elif op[0] == "advance":
            assert work == op[1], op
            fwd += op[2] - op[1]
            work = op[2]
        elif op[0] == "store":
            assert work == op[2]
            mem[op[1]] = work
        elif op[0] == "adjoint":
            assert work == op[1]
            order.append(op[1])
    return order, fwd


class Rollout:
    """n steps of a grid from (u0, body0), differentiable through revolve + fs_step_adjoint.

    Keeps `slots` device copies of the state; slots=None takes as many as half of
    the free device memory holds, up to one per step (no recomputation at all:
    500 steps of a 128^3 FP32 field are 12.6 GB), and on RK3 grids without a body
    also each step's two stage states when they fit (fs_step_record /
    fs_step_adjoint_recorded: not even the stages are recomputed).  The forward pass already keeps
    the states the schedule stores before its first adjoint, so a backward after
    a forward starts reversing at once.  Forces of every step (FSI grids) are
    recorded on the device so losses may depend on them.
    """

    def __init__(self, grid, dt, nsteps, slots=None):
        self.g = grid
        self.dt = float(dt)
        self.n = int(nsteps)
        self.slots = None if slots is None else max(1, int(slots))
        self.used_slots = self.slots
        self.recomputed = 0
        self.recorded = False
        self._kept = None

    def _recordable(self, u, body):
        """RK3 grids without a body keep, when memory allows, every step's state and its two
        stage states: the reverse sweep then recomputes nothing of any step."""
        g = self.g
        if self.slots is not None or g.scheme != F.RK3 or g.has_body or g.has_boxes or g.les_cs > 0.0:
            return False
        free, _ = torch.cuda.mem_get_info(u[0].device)
        per = sum(x.numel() * x.element_size() for x in u)
        return 3 * per * self.n <= 0.5 * free

    def _clone(self, u, body):
        return [x.clone() for x in u], (body.clone() if body is not None else None)

    def _slots_for(self, u, body):
        if self.slots is not None:
            return self.slots
        free, _ = torch.cuda.mem_get_info(u[0].device)
        per = sum(x.numel() * x.element_size() for x in u) + (body.numel() * body.element_size() if body is not None else 0)
        return max(2, min(self.n, int(0.5 * free) // max(per, 1)))

    def forward(self, u0, body0=None):
        u, body = self._clone(u0, body0)
        if self._recordable(u, body):
            tape = []
            for t in range(self.n):
                un = [x.clone() for x in u]
                v1 = [torch.empty_like(x) for x in u]
                v2 = [torch.empty_like(x) for x in u]
                self.g.step_record(u, self.dt, v1, v2)
                tape.append((un, v1, v2))
            self.recorded = True
            self.used_slots = self.n
            self._kept = ("tape", tape)
            return u, None, None
        self.recorded = False
        slots = self._slots_for(u, body)
        self.used_slots = slots
        stores, _ = split_schedule(self.n, slots)
        mem = {0: self._clone(u0, body0)}
        work = None
        forces = None
        if self.g.has_body:
            forces = torch.zeros((self.n, 3), dtype=torch.float64, device=u[0].device)
        for t in range(self.n):
            if t == self.n - 1:
                work = self._clone(u, body)
            self.g.step(u, self.dt, 1, body=body)
            if forces is not None:
                self.g.forces_device(forces[t])
            if t + 1 in stores:
                mem[stores[t + 1]] = self._clone(u, body)
        self._kept = (mem, work, slots)
        return u, body, forces

    def backward(self, u0, body0, lam_u, lam_body=None, lam_forces=None, g_body_force=None, g_stiffness=None):
        """lam_* are the adjoints of the outputs; returns (lam_u0, lam_body0).  Parameter gradients
        are accumulated into the given device tensors.  Right after forward() the states it kept
        are used (u0 and body0 must be the forward's inputs); otherwise the schedule starts from
        (u0, body0)."""
        if self._kept is not None and self._kept[0] == "tape":
            tape = self._kept[1]
            self._kept = None
            lam = [x.clone() for x in lam_u]
            self.recomputed = 0
            for t in range(self.n - 1, -1, -1):
                un, v1, v2 = tape[t]
                self.g.step_adjoint_recorded(un, v1, v2, lam, self.dt, g_body_force=g_body_force)
            return lam, None
        if self._kept is not None:
            mem, (work_u, work_b), slots = self._kept
            self._kept = None
            ops = split_schedule(self.n, slots)[1]
        else:
            slots = self._slots_for(u0, body0)
            mem = {0: self._clone(u0, body0)}
            work_u, work_b = None, None
            ops = revolve_schedule(self.n, slots)
        self.used_slots = slots
        lam = [x.clone() for x in lam_u]
        if lam_forces is not None:
            lam_forces = lam_forces.to(device=lam[0].device, dtype=torch.float64).contiguous()
        lb = lam_body.clone() if lam_body is not None else (
            torch.zeros(4, dtype=torch.float64, device=lam[0].device) if self.g.has_body else None)
        self.recomputed = 0
        for op in ops:
            if op[0] == "load":
                su, sb = mem[op[1]]
                if work_u is None:
                    work_u, work_b = self._clone(su, sb)
                else:
                    for w, s in zip(work_u, su):
                        w.copy_(s)
                    if sb is not None:
                        work_b.copy_(sb)
            elif op[0] == "advance":
                self.g.step(work_u, self.dt, op[2] - op[1], body=work_b)
                self.recomputed += op[2] - op[1]
            elif op[0] == "store":
                mem[op[1]] = self._clone(work_u, work_b)
            elif op[0] == "adjoint":
                t = op[1]
                # the force sensitivity of step t stays on the device (no host read per step)
                dJdF = lam_forces[t, :2] if lam_forces is not None else None
                self.g.step_adjoint(work_u, lam, self.dt, body_n=work_b, lam_body=lb, dJdF=dJdF,
                                    g_body_force=g_body_force, g_stiffness=g_stiffness)
        return lam, lb


class FsRollout(torch.autograd.Function):
    """u_T, body_T, forces = FsRollout.apply(grid, dt, nsteps, slots, body_force, stiffness, body0, *u0).

    body_force: float64 device tensor (ny) or None; stiffness: 1-element float64 tensor or None.
    Gradients flow to u0, body0, body_force and stiffness.
    """

    @staticmethod
    def forward(ctx, grid, dt, nsteps, slots, body_force, stiffness, body0, *u0):
        if body_force is not None:
            grid.set_body_force(body_force.detach())
        if stiffness is not None:
            grid.set_stiffness(float(stiffness.detach().reshape(-1)[0]))
        ro = Rollout(grid, dt, nsteps, slots)
        uT, bT, forces = ro.forward([x.detach() for x in u0], body0.detach() if body0 is not None else None)
        ctx.ro = ro
        ctx.has_bf = body_force is not None
        ctx.has_k = stiffness is not None
        ctx.save_for_backward(*( [x.detach() for x in u0] + ([body0.detach()] if body0 is not None else []) ))
        ctx.has_body = body0 is not None
        dummy = torch.zeros(0, device=uT[0].device)
        return tuple(uT) + (bT if bT is not None else dummy, forces if forces is not None else dummy)

    @staticmethod
    def backward(ctx, *grads):
        ro = ctx.ro
        saved = ctx.saved_tensors
        dim = ro.g.dim
        u0 = list(saved[:dim])
        body0 = saved[dim] if ctx.has_body else None
        lam_u = [g if g is not None else torch.zeros_like(x) for g, x in zip(grads[:dim], u0)]
        lam_b = grads[dim] if ctx.has_body and grads[dim] is not None and grads[dim].numel() else None
        lam_f = grads[dim + 1] if ro.g.has_body and grads[dim + 1] is not None and grads[dim + 1].numel() else None
        dev = u0[0].device
        gbf = torch.zeros(ro.g.n[1], dtype=torch.float64, device=dev) if ctx.has_bf else None
        gk = torch.zeros(1, dtype=torch.float64, device=dev) if ctx.has_k else None
        lam, lb = ro.backward(u0, body0, lam_u, lam_b, lam_f, gbf, gk)
        return (None, None, None, None, gbf, gk, lb if ctx.has_body else None) + tuple(lam)


def rollout(grid, u0, dt, nsteps, slots=None, body0=None, body_force=None, stiffness=None):
    """Differentiable rollout: returns (u_T list, body_T or empty, forces (nsteps, 3) or empty)."""
    out = FsRollout.apply(grid, dt, nsteps, slots, body_force, stiffness, body0, *u0)
    return list(out[:grid.dim]), out[grid.dim], out[grid.dim + 1]
