"""Host logic of the binomial checkpointing schedule (no GPU)."""
from math import comb

import pytest

from paper_2505_23940_b300.autodiff import revolve_schedule, simulate, split_schedule


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 64, 200])
@pytest.mark.parametrize("slots", [1, 2, 3, 5, 8])
def test_schedule_reverses_every_step_in_order(n, slots):
    order, fwd = simulate(n, slots)
    assert order == list(range(n - 1, -1, -1))
    used = {op[1] for op in revolve_schedule(n, slots) if op[0] in ("store", "load")}
    assert used <= set(range(slots))


@pytest.mark.parametrize("n,slots", [(20, 3), (64, 4), (200, 5), (1000, 6)])
def test_recomputation_within_binomial_bound(n, slots):
    """With s snapshots and t sweeps beta(s, t) = C(s + t, s) steps are reversible with at
    most t * n recomputed steps (Griewank 1992)."""
    _, fwd = simulate(n, slots)
    s = slots - 1
    t = 1
    while comb(s + t, s) < n:
        t += 1
    assert fwd <= t * n


def test_single_slot_is_quadratic_recompute():
    _, fwd = simulate(10, 1)
    assert fwd == sum(range(10))


@pytest.mark.parametrize("n", [1, 2, 5, 20, 64])
@pytest.mark.parametrize("slots", [1, 2, 3, 8, 64])
def test_split_schedule_after_a_storing_forward_pass(n, slots):
    """A forward pass that keeps the prefix's stored states and the state at n - 1 can run the
    rest of the schedule: every load finds its state, every adjoint its step, in reverse order;
    with one slot per step nothing is recomputed."""
    stores, rest = split_schedule(n, slots)
    assert rest[0] == ("adjoint", n - 1)
    assert all(0 < step < n for step in stores) and set(stores.values()) <= set(range(1, slots))
    mem = {0: 0}
    mem.update({slot: step for step, slot in stores.items()})
    work, order, fwd = n - 1, [], 0
    for op in rest:
        if op[0] == "load":
            assert mem.get(op[1]) == op[2], op
            work = op[2]
        elif op[0] == "advance":
            assert work == op[1]
            fwd += op[2] - op[1]
            work = op[2]
        elif op[0] == "store":
            assert work == op[2]
            mem[op[1]] = work
        else:
            assert work == op[1]
            order.append(op[1])
    assert order == list(range(n - 1, -1, -1))
    _, full = simulate(n, slots)
    assert fwd <= full
    if slots >= n:
        assert fwd == 0
