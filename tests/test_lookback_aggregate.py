"""The binning kernel's look-back with span aggregates, modelled on the CPU.

Beyond the paper's N/L/G counters (Section 3, Figures 6-7), a tile whose walk
has passed m preceding tiles without reaching a G counter may publish
(A, span m + 1, sum of those m + 1 counts); a later walk that reads it adds the
span's sum and continues below the span. This file checks that extension the
way the paper's protocol is checked in the oracle's model: every interleaving
of the tiles' atomic steps (small cases), and random schedules (larger ones),
end with every counter holding (G, inclusive prefix), and no schedule gets
stuck. Each walker may or may not publish an aggregate after each read that
moved it, which covers the kernel's choice of publishing once per round.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

N, L, A, G = 0, 1, 3, 2
MAX_SPAN = 64


def _steps(counts, counters, progs):
    """Every state reachable in one atomic step of one tile."""
    out = []
    for t, prog in enumerate(progs):
        kind = prog[0]
        if kind == "done":
            continue
        c = list(counters)
        p = list(progs)
        if kind == "pub_l":
            c[t] = (L, counts[t], 1)
            p[t] = ("look", t - 1, 0) if t > 0 else ("pub_g", counts[t])
            out.append((tuple(c), tuple(p)))
        elif kind == "look":
            _, k, acc = prog
            status, value, span = counters[k]
            if status == N:
                continue  # a wait, not a step
            acc += value
            nk = k - span if status == A else k - 1
            if status == G or nk < 0:
                p[t] = ("pub_g", acc + counts[t])
                out.append((tuple(c), tuple(p)))
            else:
                # the walk moved: go on, or first publish the aggregate of
                # this tile and the t - 1 - nk tiles passed
                p[t] = ("look", nk, acc)
                out.append((tuple(c), tuple(p)))
                span_here = t - nk
                if span_here <= MAX_SPAN:
                    c2 = list(counters)
                    c2[t] = (A, acc + counts[t], span_here)
                    out.append((tuple(c2), tuple(p)))
        elif kind == "pub_g":
            c[t] = (G, prog[1], 1)
            p[t] = ("done",)
            out.append((tuple(c), tuple(p)))
    return out


def explore(counts):
    g = len(counts)
    start = (tuple((N, 0, 1) for _ in range(g)), tuple(("pub_l",) for _ in range(g)))
    seen = {start}
    stack = [start]
    finals, stuck = set(), False
    while stack:
        counters, progs = stack.pop()
        nxt = _steps(counts, counters, progs)
        if not nxt:
            if all(p[0] == "done" for p in progs):
                finals.add(tuple((s, v) for s, v, _ in counters))
            else:
                stuck = True
            continue
        for st in nxt:
            if st not in seen:
                seen.add(st)
                stack.append(st)
    return finals, stuck


def run_random(counts, rng):
    g = len(counts)
    counters = tuple((N, 0, 1) for _ in range(g))
    progs = tuple(("pub_l",) for _ in range(g))
    for _ in range(100000):
        nxt = _steps(counts, counters, progs)
        if not nxt:
            break
        counters, progs = nxt[rng.randrange(len(nxt))]
    assert all(p[0] == "done" for p in progs), "schedule stuck"
    return tuple((s, v) for s, v, _ in counters)


@pytest.mark.parametrize("counts", [(3,), (2, 5), (4, 0, 7), (1, 2, 3, 4), (0, 0, 5, 0), (6, 1, 0, 2)])
def test_every_interleaving_ends_with_inclusive_prefixes(counts):
    finals, stuck = explore(list(counts))
    assert not stuck
    assert finals == {tuple((G, int(v)) for v in np.cumsum(counts))}


def test_figure7_counts_every_interleaving():
    # the five tiles of the paper's Figure 7 (inclusive prefixes 11, 26, 35, 45, 53)
    counts = [11, 15, 9, 10, 8]
    finals, stuck = explore(counts)
    assert not stuck
    assert finals == {tuple((G, v) for v in (11, 26, 35, 45, 53))}


@pytest.mark.parametrize("seed", range(20))
def test_random_schedules_on_longer_chains(seed):
    rng = random.Random(seed)
    g = rng.randint(6, 40)
    counts = [rng.randint(0, 6144) for _ in range(g)]
    for _ in range(5):
        assert run_random(counts, rng) == tuple((G, int(v)) for v in np.cumsum(counts))


def test_a_walk_jumps_a_published_span():
    # tile t's aggregate covers tiles 0..t: a walk from the last tile that
    # reads it adds the whole prefix in one read
    counts = list(range(1, 13))
    counters = [(A, int(v), t + 1) for t, v in enumerate(np.cumsum(counts))]
    k, total, reads = len(counts) - 1, 0, 0
    while k >= 0:
        s, v, span = counters[k]
        total += v
        reads += 1
        k = k - span if s == A else k - 1
    assert reads == 1 and total == sum(counts)


def test_a_wrong_span_is_caught():
    # a walk that resumed one tile too high after a span (counting its first
    # tile twice) must fail the interleaving check
    global _steps
    good = _steps

    def off_by_one(counts, counters, progs):
        out = []
        for c, p in good(counts, counters, progs):
            p = list(p)
            for t, prog in enumerate(p):
                old = progs[t]
                if prog[0] == "look" and old[0] == "look" and counters[old[1]][0] == A:
                    p[t] = ("look", prog[1] + 1, prog[2]) if prog[1] + 1 < t else prog
            out.append((c, tuple(p)))
        return out

    try:
        _steps = off_by_one
        finals, _ = explore([1, 2, 3, 4])
    finally:
        _steps = good
    assert finals != {tuple((G, int(v)) for v in np.cumsum([1, 2, 3, 4]))}


# ---------------------------------------------------------------------------
# The kernel's own round structure: a round issues reads of up to W preceding
# counters (each read is its own atomic step, so the reads of one round may
# see different moments), then folds them in order exactly as the kernel's
# consume() does - stop at an N, after an aggregate skip the window's
# remaining rows - and publishes an aggregate after a round that moved, or G
# once done. Checked: every terminal state holds the inclusive prefixes, and a
# terminal state stays reachable from every reachable state (no livelock).

W = 4


def _kernel_steps(counts, counters, progs):
    out = []
    for t, prog in enumerate(progs):
        kind = prog[0]
        if kind == "done":
            continue
        c = list(counters)
        p = list(progs)
        if kind == "pub_l":
            c[t] = (G, counts[t], 1) if t == 0 else (L, counts[t], 1)
            p[t] = ("done",) if t == 0 else ("read", t, 0, ())
        elif kind == "read":
            _, left, exclusive, got = prog
            w = len(got)
            # rows before the chain's first tile read as (G, 0), as in issue()
            val = counters[left - 1 - w] if w < left else (G, 0, 1)
            got = got + (val,)
            if len(got) < W:
                p[t] = ("read", left, exclusive, got)
            else:
                left0, done = left, False
                for s, v, span in got:
                    if done or s == N:
                        break
                    if s == A:
                        exclusive += v
                        left -= span
                        done = left == 0
                        break
                    exclusive += v
                    left -= 1
                    done = s == G or left == 0
                if done:
                    p[t] = ("pub_g", exclusive + counts[t])
                elif left != left0 and t - left + 1 <= MAX_SPAN:
                    p[t] = ("pub_a", left, exclusive)
                else:
                    p[t] = ("read", left, exclusive, ())
        elif kind == "pub_a":
            _, left, exclusive = prog
            c[t] = (A, exclusive + counts[t], t - left + 1)
            p[t] = ("read", left, exclusive, ())
        elif kind == "pub_g":
            c[t] = (G, prog[1], 1)
            p[t] = ("done",)
        out.append((tuple(c), tuple(p)))
    return out


def _explore_kernel(counts):
    g = len(counts)
    start = (tuple((N, 0, 1) for _ in range(g)), tuple(("pub_l",) for _ in range(g)))
    succ = {}
    stack = [start]
    while stack:
        st = stack.pop()
        if st in succ:
            continue
        nxt = _kernel_steps(counts, *st)
        succ[st] = nxt
        stack.extend(n for n in nxt if n not in succ)
    terminal = {s for s, n in succ.items() if not n}
    # states from which a terminal state is reachable (reverse reachability)
    pred = {s: [] for s in succ}
    for s, n in succ.items():
        for x in n:
            pred[x].append(s)
    good, work = set(terminal), list(terminal)
    while work:
        x = work.pop()
        for y in pred[x]:
            if y not in good:
                good.add(y)
                work.append(y)
    finals = {tuple((s, v) for s, v, _ in st[0]) for st in terminal}
    return finals, len(good) == len(succ), len(succ)


@pytest.mark.parametrize("counts", [(5,), (2, 3), (1, 0, 4), (3, 1, 2, 6), (0, 7, 0, 2)])
def test_kernel_rounds_every_interleaving(counts):
    finals, live, states = _explore_kernel(list(counts))
    assert live, "a reachable state cannot finish"
    assert finals == {tuple((G, int(v)) for v in np.cumsum(counts))}
    assert states > len(counts)


def test_kernel_rounds_fold_a_stale_window_correctly():
    # a round whose first row is an aggregate skips the rows read after it,
    # whatever they held when read: a wrong skip (one row too few) is caught
    global _kernel_steps
    good = _kernel_steps

    def skip_one_short(counts, counters, progs):
        out = []
        for c, p in good(counts, counters, progs):
            p = list(p)
            for t, (old, new) in enumerate(zip(progs, p)):
                if old[0] == "read" and len(old[3]) == W - 1 and new[0] in ("read", "pub_a"):
                    got = old[3] + (counters[old[1] - 1 - (W - 1)] if W - 1 < old[1] else (G, 0, 1),)
                    if got[0][0] == A and new[1] < old[1] - 1:
                        p[t] = (new[0], new[1] + 1) + tuple(new[2:])
            out.append((c, tuple(p)))
        return out

    try:
        _kernel_steps = skip_one_short
        finals, _, _ = _explore_kernel([1, 2, 3, 4])
    finally:
        _kernel_steps = good
    assert finals != {tuple((G, int(v)) for v in np.cumsum([1, 2, 3, 4]))}
