"""Host logic of the binomial checkpointing schedule (no GPU)."""
from math import comb

import pytest

from paper_2505_23940_b300.autodiff import revolve_schedule, simulate


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
