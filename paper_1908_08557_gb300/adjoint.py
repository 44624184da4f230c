"""Gradients of a loss on the final state of an N-step driven run with
respect to the driver magnetogram B_z and the driver velocity snapshots
v0, v1, through the library's hand-written adjoint step.

* `optimal_splits`, `Revolver`: checkpointing by the treeverse recursion
  of Griewank 1992 ("Achieving logarithmic growth of temporal and spatial
  complexity in reverse automatic differentiation"): with s free checkpoint
  slots an interval is split at a checkpoint, the right part reversed with
  s - 1 slots, then the left part with s.  The split points are the ones a
  dynamic program over (length, slots) finds to minimise the recomputed
  steps: for the intervals that end at the last step the checkpoints are
  taken during the forward sweep at no cost, for the others every step
  advanced counts.  (`binomial_split`, the repetition-number rule, serves
  runs too long for the program.)
* `DrivenRun`: a torch.autograd.Function (B_z, v0, v1) -> final state.
* `BzPlane`: B_z on one layer of a state, with its transpose, for misfit
  losses (the adjoint workload's loss is the L2 misfit of B_z at one height).

All arithmetic runs in libmhd; this module schedules calls and holds the
checkpoint buffers (torch device memory).
"""
from __future__ import annotations

from functools import lru_cache
from math import comb
from typing import Dict, List, Optional

import torch


def binomial_split(l: int, s: int) -> int:
    """Length of the left part when reversing l > 1 steps with s >= 1 slots:
    with t the smallest repetition number for which C(s + t, s) >= l, the
    right part gets at most C(s - 1 + t, s - 1) steps (reversed with s - 1
    slots), the left part the rest (at least 1, at most l - 1)."""
    t = 0
    while comb(s + t, s) < l:
        t += 1
    right = comb(s - 1 + t, s - 1)
    left = max(1, l - right)
    return min(left, l - 1)


# the split program runs for steps x slots up to this (host time ~ 2 s);
# longer runs take the repetition-number rule
DP_MAX_WORK = 120_000


@lru_cache(maxsize=8)
def optimal_splits(n: int, slots: int):
    """Minimal recomputation of reversing up to n steps with up to `slots`
    free checkpoint slots, and the first split of each subproblem.

    T[l, s]: steps advanced to reverse l steps from a checkpoint at their
    start (no live state): 0 for l = 1; l (l - 1) / 2 with no slot (every
    step recomputed from the start); else min over m of m (advance and save)
    + T[l - m, s - 1] (the right part) + T[m, s] (the left part, its slot
    back).  R[l, s]: the same when the checkpoints of the first pass are
    taken during the forward sweep: min over m of R[l - m, s - 1] + T[m, s].
    Returns (T, R, mT, mR), mT and mR the minimising m (the smallest on
    ties).  Cached per (n, slots): a gradient loop plans once."""
    import numpy as np
    S = max(0, min(slots, n - 1))
    T = np.zeros((n + 1, S + 1), dtype=np.int64)
    R = np.zeros((n + 1, S + 1), dtype=np.int64)
    mT = np.ones((n + 1, S + 1), dtype=np.int64)
    mR = np.ones((n + 1, S + 1), dtype=np.int64)
    ll = np.arange(n + 1, dtype=np.int64)
    T[:, 0] = np.maximum(ll * (ll - 1) // 2, 0)
    R[:, 0] = T[:, 0]
    for s in range(1, S + 1):
        for L in range(2, n + 1):
            m = np.arange(1, L, dtype=np.int64)
            c = m + T[L - m, s - 1] + T[m, s]
            k = int(np.argmin(c))
            T[L, s], mT[L, s] = c[k], k + 1
        for L in range(2, n + 1):
            m = np.arange(1, L, dtype=np.int64)
            c = R[L - m, s - 1] + T[m, s]
            k = int(np.argmin(c))
            R[L, s], mR[L, s] = c[k], k + 1
    return T, R, mT, mR


class Revolver:
    """Forward sweep with checkpoints and the reverse sweep over them.

    `slots` checkpoints of the state fit the memory budget (besides the
    initial one).  When the whole history fits as tapes -- three substep
    states per step, i.e. 3 n checkpoints for n steps -- the forward sweep
    keeps every step's tape and the reverse sweep reads them back: no forward
    substep is recomputed.  Otherwise the checkpoints are placed by the
    split program and the reverse sweep recomputes from them."""

    def __init__(self, sim, slots: int):
        if slots < 0:
            raise ValueError("slots >= 0")
        self.sim = sim
        self.slots = slots
        self.pool: List[torch.Tensor] = []
        self.tapes: List[torch.Tensor] = []
        self.free = list(range(1, slots + 1))
        self.forward_steps = 0      # steps taken in the forward sweep
        self.recomputed_steps = 0   # steps recomputed during the reverse sweep
        self.adjoint_steps = 0

    def _split(self, i0: int, i1: int, s: int) -> int:
        """Checkpoint position inside [i0, i1) with s free slots; intervals
        that end at the last step are on the forward sweep's chain."""
        l = i1 - i0
        if self.mT is None:
            return i0 + binomial_split(l, s)
        tab = self.mR if i1 == self.n else self.mT
        return i0 + int(tab[l, min(s, tab.shape[1] - 1)])

    def _chain(self, n: int) -> List[int]:
        out, i0, s = [], 0, self.slots
        while n - i0 > 1 and s > 0:
            m = self._split(i0, n, s)
            out.append(m)
            i0, s = m, s - 1
        return out

    def taped(self, nsteps: int) -> bool:
        """The whole history of nsteps fits as tapes."""
        return nsteps >= 1 and 3 * nsteps <= self.slots + 1

    def forward(self, nsteps: int):
        """From the current state (time t0), take nsteps, saving the tapes
        or the checkpoints the reverse sweep starts from."""
        sim = self.sim
        self.n = nsteps
        if self.taped(nsteps):
            self.tapes = [sim.new_tape() for _ in range(nsteps)]
            for tp in self.tapes:
                sim.step_taped(tp)
            self.forward_steps += nsteps
            return
        self.tapes = []
        if not self.pool:
            self.pool = [sim.new_checkpoint() for _ in range(self.slots + 1)]
        self.mT = self.mR = None
        if nsteps > 1 and nsteps * min(self.slots, nsteps - 1) <= DP_MAX_WORK:
            _, _, self.mT, self.mR = optimal_splits(nsteps, self.slots)
        self.t_start = sim.save(self.pool[0])
        self.saved: Dict[int, tuple] = {}
        pos = 0
        for m in self._chain(nsteps):
            sim.step(m - pos)
            slot = self.free.pop()
            self.saved[m] = (slot, sim.save(self.pool[slot]))
            pos = m
        sim.step(nsteps - pos)
        self.forward_steps += nsteps

    def reverse(self):
        """Reverse sweep over the forward run; the adjoint must have been
        seeded with mhd_adjoint_init."""
        if self.tapes:
            for tp in reversed(self.tapes):
                self.sim.adjoint_step_taped(tp)
                self.adjoint_steps += 1
            return
        self._rev(0, self.n, (0, self.t_start), self.slots)

    def _rev(self, i0: int, i1: int, ck, s: int):
        """Reverse steps i0 .. i1-1 starting from checkpoint ck with s free
        slots: split at m (`_split`), reverse the right part with s - 1
        slots from a checkpoint at m, release that slot, then reverse the left
        part.  An explicit stack keeps that order without recursion (one
        level per slot would exceed Python's recursion limit for large slot
        counts)."""
        sim = self.sim
        stack = [("rev", i0, i1, ck, s)]
        while stack:
            item = stack.pop()
            if item[0] == "free":
                self.free.append(item[1])
                continue
            _, i0, i1, ck, s = item
            slot0, t0 = ck
            if i1 - i0 == 1:
                sim.restore(self.pool[slot0], t0)
                sim.adjoint_step()
                self.adjoint_steps += 1
                continue
            if s == 0:
                for j in range(i1 - 1, i0 - 1, -1):
                    sim.restore(self.pool[slot0], t0)
                    if j > i0:
                        sim.step(j - i0)
                        self.recomputed_steps += j - i0
                    sim.adjoint_step()
                    self.adjoint_steps += 1
                continue
            m = self._split(i0, i1, s)
            if m in self.saved:
                ckm = self.saved.pop(m)
            else:
                sim.restore(self.pool[slot0], t0)
                sim.step(m - i0)
                self.recomputed_steps += m - i0
                slot = self.free.pop()
                ckm = (slot, sim.save(self.pool[slot]))
            stack.append(("rev", i0, m, ck, s))
            stack.append(("free", ckm[0]))
            stack.append(("rev", m, i1, ckm, s - 1))


class DrivenRun(torch.autograd.Function):
    """(bz, v0, v1, state0) -> state after `nsteps` steps from `state0` at
    t = 0; gradients for the driver (B_z, v0, v1) and, when state0 requires
    one, for the initial state (the adjoint of the initial state, the
    stateful ghost layers folded onto the photosphere).  The handle must have
    been created with adjoint=True and dt_fixed > 0."""

    @staticmethod
    def forward(ctx, bz, v0, v1, sim, state0, nsteps: int, slots: int, t0: float = 0.0, t1: float = 1.0):
        sim.set_driver(bz.detach().contiguous(), v0.detach().contiguous(), v1.detach().contiguous(), t0, t1)
        sim.write(state0.detach().contiguous())
        sim.set_time(0.0)
        rv = Revolver(sim, slots)
        rv.forward(nsteps)
        ctx.sim, ctx.rv = sim, rv
        return sim.read()

    @staticmethod
    def backward(ctx, gstate):
        sim, rv = ctx.sim, ctx.rv
        sim.adjoint_init(gstate.contiguous())
        rv.reverse()
        g = sim.adjoint_read()
        gs = g["lam"] if ctx.needs_input_grad[4] else None
        return g["bz"], g["v0"], g["v1"], None, gs, None, None, None, None


class BzPlane(torch.autograd.Function):
    """state [8, nz, ny, nx] -> B_z = D1x A_y - D1y A_x on layer k."""

    @staticmethod
    def forward(ctx, state, sim, k: int):
        ctx.sim, ctx.k = sim, k
        return sim.bz_plane(state.detach(), k)

    @staticmethod
    def backward(ctx, gbz):
        return ctx.sim.bz_plane_adjoint(gbz, ctx.k), None, None
