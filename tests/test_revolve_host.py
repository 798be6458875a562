"""Binomial checkpointing schedules (host logic, no GPU): the planner's cost
is optimal (exhaustive search over every checkpointing strategy on small
cases), matches its closed-form corners, and the emitted action list is a
valid schedule that attains it."""
import heapq
import itertools

import pytest

import paper_1603_03971_gb300 as rtm


def _exhaustive_cost(n, s):
    """Fewest forward steps to deliver states n, n-1, ..., 1 in that order from
    the free initial state 0 with s slots: Dijkstra over (next state to
    deliver, working state, set of stored states). Moves: advance the working
    state by one (cost 1), store it, drop a stored state, restore a stored
    state or state 0 into the working pair (cost 0), deliver the next state
    when the working pair or a slot holds it (cost 0)."""
    start = (n, 0, frozenset())
    dist = {start: 0}
    heap = [(0, start)]
    while heap:
        d, (nxt, w, slots) = heapq.heappop(heap)
        if nxt == 0:
            return d
        if d > dist.get((nxt, w, slots), 1 << 60):
            continue
        moves = []
        if w < nxt:
            moves.append((1, (nxt, w + 1, slots)))
        if len(slots) < s and w not in slots and w > 0:
            moves.append((0, (nxt, w, slots | {w})))
        for q in slots:
            moves.append((0, (nxt, w, slots - {q})))
            moves.append((0, (nxt, q, slots)))
        moves.append((0, (nxt, 0, slots)))
        if w == nxt or nxt in slots:
            moves.append((0, (nxt - 1, w, slots)))
        for c, st in moves:
            if d + c < dist.get(st, 1 << 60):
                dist[st] = d + c
                heapq.heappush(heap, (d + c, st))
    raise AssertionError("unreachable")


@pytest.mark.parametrize("n,s", [(n, s) for n in range(1, 8) for s in range(0, 4)])
def test_cost_is_optimal(n, s):
    assert rtm.revolve_cost(n, s) == _exhaustive_cost(n, s)


def test_cost_corners():
    for n in (1, 5, 40, 300):
        assert rtm.revolve_cost(n, 0) == n * (n + 1) // 2
        assert rtm.revolve_cost(n, n) == n  # one sweep, every state kept
        assert rtm.revolve_cost(n, n + 7) == n
    assert rtm.revolve_cost(0, 3) == 0
    # more slots never cost more
    for n in (30, 97):
        costs = [rtm.revolve_cost(n, s) for s in range(0, 12)]
        assert all(a >= b for a, b in zip(costs, costs[1:]))
    assert rtm.revolve_cost(200000, 100) == -1  # beyond the planning limit


def _simulate(n, s, actions):
    """Replays the actions: returns the forward steps taken; asserts that
    every state is delivered once, in order n..1, from where the action says
    it is, and that no more than s slots are ever in use."""
    work, slots, steps, expect = None, {}, 0, n  # the working pair starts unknown
    for op, a, b, c in actions:
        if op == 0:  # restore
            if a < 0:
                work = 0
            else:
                assert slots.get(a) == b
                work = b
            assert work == b
        elif op == 1:  # advance
            assert work is not None and work == a and b > a
            steps += b - a
            work = b
        elif op == 2:  # store
            assert a not in slots and 0 <= a < s and work is not None and work == b
            slots[a] = b
        elif op == 3:  # deliver
            assert a == expect
            if b < 0:
                assert work is not None and work == a
            else:
                assert slots.get(b) == a
            expect -= 1
        elif op == 4:  # free
            assert a in slots
            del slots[a]
        else:
            raise AssertionError(op)
        assert len(slots) <= s
    assert expect == 0
    return steps


@pytest.mark.parametrize("n,s", [(1, 0), (17, 0), (5, 10), (50, 1), (50, 3), (200, 10),
                                 (750, 20), (2000, 40)])
def test_schedule_is_valid_and_attains_the_cost(n, s):
    acts = rtm.revolve_schedule(n, s)
    assert _simulate(n, s, acts) == rtm.revolve_cost(n, s)
