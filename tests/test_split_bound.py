"""CPU checks of the bounds behind the split refinement scans' workspace.

The refinement orders its p-tiles by an estimated cost; with `slots`
resident CTAs and total cost W, a p-tile costing c with c * slots > W is
scanned by K = min(8, ceil(2 c slots / W)) CTAs (parts), every other p-tile
by one. The library sizes the order arrays for 2 * slots extra entries and
the split records for `slots` split p-tiles (148 SMs x 9 CTAs at most), and
launches 2 * slots extra blocks. This file restates the rule and checks
that no cost distribution exceeds those bounds: K - 1 < 2 c slots / W sums
to less than 2 slots, and fewer than `slots` p-tiles can each cost more than
W / slots."""
import numpy as np
import pytest

SLOTS_MAX = 148 * 9


def parts(c, total, slots):
    if total == 0 or c * slots <= total:
        return 1
    return min(8, -(-2 * c * slots // total))


def check(costs, slots):
    costs = [int(c) for c in costs]
    total = sum(costs)
    ks = [parts(c, total, slots) for c in costs]
    extra = sum(k - 1 for k in ks)
    split = sum(1 for k in ks if k > 1)
    assert extra < 2 * slots or extra == 0
    assert split < slots or split == 0
    assert extra <= 2 * SLOTS_MAX and split <= 2 * SLOTS_MAX
    return extra, split


@pytest.mark.parametrize("slots", [148 * 5, 148 * 6, 148 * 7, SLOTS_MAX])
def test_bounds_on_random_and_extreme_costs(slots):
    rng = np.random.default_rng(slots)
    for _ in range(200):
        t = int(rng.integers(1, 40000))
        kind = rng.integers(0, 4)
        if kind == 0:
            costs = rng.integers(0, 1025, size=t)
        elif kind == 1:                                  # heavy tail
            costs = np.minimum(1024, (rng.pareto(1.2, size=t) * 20).astype(np.int64))
        elif kind == 2:                                  # a few huge p-tiles
            costs = np.zeros(t, dtype=np.int64)
            costs[rng.choice(t, size=min(t, 5), replace=False)] = 1024
        else:                                            # equal costs
            costs = np.full(t, int(rng.integers(0, 1025)))
        check(costs, slots)
    # one p-tile holds all the cost: it alone splits, into the cap of 8
    extra, split = check([1024] + [0] * 999, slots)
    assert (extra, split) == (7, 1)
    # as many p-tiles as slots with equal cost: nobody exceeds the span
    assert check([100] * slots, slots) == (0, 0)


def test_split_rule_matches_the_span_reading():
    """A p-tile splits only when its cost exceeds the mean load of a slot,
    into about twice as many parts as it has slots' worth of cost."""
    slots, total = 100, 100000          # span = 1000
    assert parts(1000, total, slots) == 1
    assert parts(1001, total, slots) == 3   # ceil(2 * 1001 / 1000)
    assert parts(2000, total, slots) == 4
    assert parts(10000, total, slots) == 8  # capped
    assert parts(5, 0, slots) == 1
