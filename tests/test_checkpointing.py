"""Host logic of the checkpointing (paper_1908_08557_gb300/adjoint.py) on
CPU, with a stand-in for the simulation handle whose state is the step
index: the reverse sweep must take the adjoint of every step exactly once,
in reverse order, each from the state at the start of that step; it must
never need more checkpoint slots than it was given; and its recomputation
must match the closed forms at the two ends of the slot range.

The split program is pinned twice from outside itself: its table for a
reversal from a bare start checkpoint against the closed form of Griewank
and Walther (2000, ACM TOMS 26, "Algorithm 799: revolve"), and both of its
tables, with the Revolver's own count, against a shortest-path search over
every schedule of checkpoint saves, deletes, restores and steps on tiny
runs."""
import heapq
from itertools import combinations
from math import comb

import pytest

pytest.importorskip("torch")

from paper_1908_08557_gb300.adjoint import Revolver, binomial_split, optimal_splits  # noqa: E402


class StepCounter:
    """The calls the scheduler makes, on a state that is just the step index."""

    def __init__(self):
        self.k = 0
        self.adjoint_at = []

    def new_checkpoint(self):
        return {}

    def save(self, buf):
        buf["k"] = self.k
        return float(self.k)

    def restore(self, buf, t):
        assert t == float(buf["k"])
        self.k = buf["k"]

    def step(self, n):
        assert n > 0
        self.k += n

    def adjoint_step(self):
        self.adjoint_at.append(self.k)

    # tapes: the substep states of one step, kept for its reverse step
    def new_tape(self):
        return {}

    def step_taped(self, tape):
        tape["k"] = self.k
        self.k += 1

    def adjoint_step_taped(self, tape):
        self.adjoint_at.append(tape["k"])


def _sweep(n, slots):
    sim = StepCounter()
    rv = Revolver(sim, slots)
    rv.forward(n)
    assert sim.k == n and rv.forward_steps == n
    rv.reverse()
    assert sim.adjoint_at == list(range(n - 1, -1, -1))
    assert rv.adjoint_steps == n
    assert sorted(rv.free) == list(range(1, slots + 1))  # every slot returned
    return rv.recomputed_steps


@pytest.mark.parametrize("n", [1, 2, 3, 7, 10, 33, 100])
@pytest.mark.parametrize("slots", [0, 1, 2, 3, 5, 10, 99])
def test_reverse_order_and_slots(n, slots):
    _sweep(n, slots)


@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_taped_history_when_it_fits(n):
    """With memory for three checkpoints per step (a tape of the three
    substep states), the forward sweep keeps every step's tape and the
    reverse sweep reads them back in reverse order: nothing is recomputed
    and no checkpoint slot is used; one slot less and the checkpoints take
    over."""
    sim = StepCounter()
    rv = Revolver(sim, 3 * n - 1)
    assert rv.taped(n)
    rv.forward(n)
    assert sim.k == n and len(rv.tapes) == n and not rv.pool
    rv.reverse()
    assert sim.adjoint_at == list(range(n - 1, -1, -1))
    assert rv.recomputed_steps == 0 and rv.adjoint_steps == n
    assert not Revolver(StepCounter(), 3 * n - 2).taped(n)


@pytest.mark.parametrize("n", [2, 10, 57, 100])
def test_recompute_closed_forms(n):
    # no slot: every step j is recomputed from the start (j steps)
    assert _sweep(n, 0) == n * (n - 1) // 2
    # a slot per step: nothing is recomputed
    assert _sweep(n, n - 1) == 0
    # more slots never cost more recomputation
    prev = None
    for s in range(0, n):
        r = _sweep(n, s)
        assert prev is None or r <= prev, (n, s, r, prev)
        prev = r


def test_binomial_split_bounds():
    for l in range(2, 200):
        for s in range(1, 12):
            m = binomial_split(l, s)
            assert 1 <= m <= l - 1


def _gw_forward_steps(l, c):
    """Minimal steps to reverse l steps with c checkpoints, the one at the
    start included (Griewank and Walther 2000): r l - C(c + r, r - 1), r the
    repetition number, the smallest with C(c + r, c) >= l (the binomial
    with a negative lower index is 0)."""
    r = 0
    while comb(c + r, c) < l:
        r += 1
    return r * l - (comb(c + r, r - 1) if r > 0 else 0)


def test_split_program_matches_the_closed_form():
    T, _, _, _ = optimal_splits(120, 9)
    for l in range(1, 121):
        for s in range(0, 10):
            assert T[l, s] == _gw_forward_steps(l, s + 1), (l, s)


def _search(n, s, forward_free):
    """Fewest steps over every schedule that reverses n steps: a state is
    (the saved step indices besides the start, the live step or -1, the
    step whose adjoint is next); moves are step the live state (cost 1),
    save it, drop a checkpoint, restore one, and take the adjoint of step j
    when the live state sits at j (the live state is spent).  With
    `forward_free` the reversal may begin from any set of at most s saves
    made during the forward sweep, at no cost; else from the start alone."""
    starts = [frozenset()]
    if forward_free:
        starts = [frozenset(c) for k in range(0, s + 1) for c in combinations(range(1, n), k)]
    dist, heap = {}, []
    for c in starts:
        key = (c, -1, n - 1)
        dist[key] = 0
        heap.append((0, key))
    heapq.heapify(heap)
    while heap:
        d, key = heapq.heappop(heap)
        if d > dist[key]:
            continue
        ck, live, j = key
        if j < 0:
            return d
        moves = []
        if live == j:
            moves.append((0, (ck, -1, j - 1)))
        if 0 <= live < j:
            moves.append((1, (ck, live + 1, j)))
            if live > 0 and live not in ck and len(ck) < s:
                moves.append((0, (ck | {live}, live, j)))
        for c in [0, *ck]:
            if c <= j:
                moves.append((0, (ck, c, j)))
        for c in ck:
            moves.append((0, (ck - {c}, live, j)))
        for w, nk in moves:
            if d + w < dist.get(nk, 1 << 60):
                dist[nk] = d + w
                heapq.heappush(heap, (d + w, nk))
    raise AssertionError("no schedule")


@pytest.mark.parametrize("n", [2, 3, 5, 8])
@pytest.mark.parametrize("slots", [1, 2, 3])
def test_split_program_and_revolver_are_optimal(n, slots):
    T, R, _, _ = optimal_splits(n, slots)
    S = min(slots, n - 1)
    assert T[n, S] == _search(n, slots, forward_free=False)
    assert R[n, S] == _search(n, slots, forward_free=True)
    assert _sweep(n, slots) == R[n, S]


def test_revolver_beats_the_repetition_number_rule():
    # the rule sizes the right part for s snapshots although s + 1 (the
    # start's among them) are live; the split program does better
    T, R, _, _ = optimal_splits(100, 10)
    assert _sweep(100, 10) == R[100, 10] == 112
