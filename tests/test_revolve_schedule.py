"""The binomial checkpointing schedule of wave_grad_revolve (host only).

* its forward-step count is the minimum over every recursive checkpoint
  placement, found here by brute force (dynamic programming over the first
  stored state), for every step count up to 40 and up to 6 slots;
* replayed on a model of the run (which step the current state holds, what
  each slot holds), every action is legal, every time index is reversed
  exactly once and in descending order, and no more than nslots slots are
  used;
* the two ends: with no slot every reversed step recomputes from step 0
  (nt (nt + 1) / 2 steps), with nt - 1 slots each step is computed twice at
  most (2 nt - 1).
"""
from functools import lru_cache

import pytest

ADVANCE, TAKESHOT, RESTORE, YOUTURN = 0, 1, 2, 3


@lru_cache(maxsize=None)
def _best(l, s):
    """Fewest forward steps (besides the one inside each reversed step) to
    reverse l steps from a held start state with s free slots: either
    recompute from the start for every step (s = 0), or advance to some
    m in [1, l), store that state, reverse [m, l) with s - 1 slots, then
    [0, m) with s."""
    if l <= 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(m + _best(l - m, s - 1) + _best(m, s) for m in range(1, l))


@pytest.mark.parametrize("nslots", range(0, 7))
def test_forward_steps_are_the_brute_force_minimum(wavelib, nslots):
    for nt in range(1, 41):
        if nslots > nt:
            continue
        assert wavelib.revolve_forward_steps(nt, nslots) == _best(nt, nslots) + nt, (nt, nslots)


def _replay(nt, nslots, sched):
    cur = 0  # the run starts at the zero state of step 0
    slots = {}
    reversed_steps = []
    forward = 0
    for kind, a, b in sched:
        if kind == ADVANCE:
            assert cur == a and a < b <= nt
            forward += b - a
            cur = b
        elif kind == TAKESHOT:
            assert cur == a and 0 <= b < nslots
            slots[b] = a
        elif kind == RESTORE:
            assert (b == -1 and a == 0) or slots.get(b) == a
            cur = a
        else:
            assert kind == YOUTURN and cur == a and 0 <= a < nt
            forward += 1
            reversed_steps.append(a)
            cur = a + 1
    assert reversed_steps == list(range(nt - 1, -1, -1))
    assert len(slots) <= nslots
    return forward


@pytest.mark.parametrize("nt,nslots", [(1, 0), (1, 1), (7, 0), (7, 2), (20, 3), (64, 4), (100, 9),
                                       (300, 5), (1000, 10), (2000, 40), (50, 49), (50, 50)])
def test_schedule_replays_legally(wavelib, nt, nslots):
    sched = wavelib.revolve_schedule(nt, nslots)
    assert _replay(nt, nslots, sched) == wavelib.revolve_forward_steps(nt, nslots)


def test_the_two_ends_and_invalid_arguments(wavelib):
    for nt in (1, 2, 9, 33):
        assert wavelib.revolve_forward_steps(nt, 0) == nt * (nt + 1) // 2
        assert wavelib.revolve_forward_steps(nt, max(nt - 1, 0)) == 2 * nt - 1
        assert wavelib.revolve_forward_steps(nt, nt) == 2 * nt - 1
    assert wavelib.revolve_forward_steps(0, 0) == -1
    assert wavelib.revolve_forward_steps(10, 11) == -1
    assert wavelib.revolve_forward_steps(10, -1) == -1
    # more slots never cost more steps
    prev = None
    for s in range(0, 30):
        f = wavelib.revolve_forward_steps(500, s)
        assert prev is None or f <= prev
        prev = f
    g = wavelib.Grid((20, 20, 20), (0.01,) * 3, 1e-3, 40, 4)
    assert wavelib.workspace_bytes(g, wavelib.WAVE_OP_REVOLVE, 1, 2, 41) == 0
    a = wavelib.workspace_bytes(g, wavelib.WAVE_OP_REVOLVE, 1, 2, 3)
    b = wavelib.workspace_bytes(g, wavelib.WAVE_OP_REVOLVE, 1, 2, 5)
    assert b - a == 2 * 2 * 4 * 20 * 20 * 24  # two more states of two z-padded levels
