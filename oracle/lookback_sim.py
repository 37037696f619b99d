"""Model of the chained-scan status-counter protocol (arXiv 2206.01784, Section 3, Figures 6-7).

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``).

One digit, g tiles. Each tile owns one counter holding (status, value) with
status N (value not ready), L (the tile's local digit count) or G (the
inclusive prefix over this and all earlier tiles). A tile's program, taken as
a sequence of atomic steps, is:

  1. publish (L, local count);
  2. look back: read the counter of the previous tile; while it is N, wait;
     if it is L, add its value and move one tile further back; if it is G, add
     its value and stop. Reaching the start of the array also stops;
  3. publish (G, accumulated + local count).

``explore`` enumerates every interleaving of these steps (a read of an N
counter is a wait, not a step) and returns the set of final counter states
together with whether any reachable state was stuck. Pure Python, meant for a
handful of tiles.
"""
from __future__ import annotations

N, L, G = 0, 1, 2


def _initial(counts):
    g = len(counts)
    counters = tuple((N, 0) for _ in range(g))
    # per-tile program state: ("pub_l",) | ("look", k, acc) | ("pub_g", value) | ("done",)
    progs = tuple(("pub_l",) for _ in range(g))
    return counters, progs


def _enabled(counts, counters, progs):
    """All successor states reachable in one atomic step."""
    out = []
    for t, prog in enumerate(progs):
        kind = prog[0]
        if kind == "done":
            continue
        c = list(counters)
        p = list(progs)
        if kind == "pub_l":
            c[t] = (L, counts[t])
            p[t] = ("look", t - 1, 0) if t > 0 else ("pub_g", counts[t])
        elif kind == "look":
            _, k, acc = prog
            status, value = counters[k]
            if status == N:
                continue  # waiting: no step
            acc += value
            if status == G or k == 0:
                p[t] = ("pub_g", acc + counts[t])
            else:
                p[t] = ("look", k - 1, acc)
        elif kind == "pub_g":
            c[t] = (G, prog[1])
            p[t] = ("done",)
        out.append((tuple(c), tuple(p)))
    return out


def explore(counts):
    """Every interleaving: (set of final counter tuples, stuck_state_seen)."""
    start = _initial(counts)
    seen = {start}
    stack = [start]
    finals = set()
    stuck = False
    while stack:
        counters, progs = stack.pop()
        nxt = _enabled(counts, counters, progs)
        if not nxt:
            if all(p[0] == "done" for p in progs):
                finals.add(counters)
            else:
                stuck = True
            continue
        for s in nxt:
            if s not in seen:
                seen.add(s)
                stack.append(s)
    return finals, stuck


def run_schedule(counts, schedule):
    """Apply steps of the tiles listed in ``schedule`` (tile ids) in order.

    Returns the list of counter states after each step. A step of a tile that
    is waiting or done raises ValueError."""
    counters, progs = _initial(counts)
    history = []
    for t in schedule:
        prog = progs[t]
        if prog[0] == "done":
            raise ValueError(f"tile {t} is done")
        succ = None
        for c, p in _enabled(counts, counters, progs):
            if p[t] != progs[t] and all(p[u] == progs[u] for u in range(len(progs)) if u != t):
                succ = (c, p)
        if succ is None:
            raise ValueError(f"tile {t} cannot step (waiting)")
        counters, progs = succ
        history.append(counters)
    return history
