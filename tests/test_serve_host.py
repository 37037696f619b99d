"""Host logic of the sort service: the device-memory arena and admission (no GPU)."""
import numpy as np

from paper_2206_01784_gb300 import serve


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(10 * 256)
    x = a.alloc(256)
    y = a.alloc(300)  # rounds to 512
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768)
    assert a.used == 1024
    assert a.alloc(7 * 256) is None       # only 6 blocks left
    a.free(y, 300)
    assert a.alloc(512) == 256            # first fit reuses the hole
    a.free(256, 512)
    a.free(x, 256)
    a.free(z, 256)
    assert a.free_list == [(0, 2560)] and a.used == 0  # everything coalesced


def test_arena_random_alloc_free_keeps_invariants():
    rng = np.random.default_rng(0)
    a = serve.Arena(1 << 20)
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.5:
            off, n = live.pop(int(rng.integers(len(live))))
            a.free(off, n)
        else:
            n = int(rng.integers(1, 20000))
            off = a.alloc(n)
            if off is not None:
                live.append((off, n))
        # blocks never overlap and the books balance
        spans = sorted([(o, serve._round(n)) for o, n in live] + a.free_list)
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2
        assert a.used == sum(serve._round(n) for _, n in live)


def _ws(kt, n, segs):
    return 1024 + 16 * n + 64 * segs


def test_admission_fifo_grouping_and_blocking():
    arena = serve.Arena(1 << 20)
    adm = serve.Admission(arena, _ws)
    reqs = [serve.Request(0, "u32", 1000, 0.0), serve.Request(1, "u64", 500, 0.1),
            serve.Request(2, "u32", 2000, 0.2), serve.Request(3, "u32", 100, 5.0)]
    for r in reqs:
        adm.arrive(r)
    out = adm.take(now=1.0)
    kinds = {kt: [r.rid for r in rs] for kt, rs, _ in out}
    assert kinds == {"u32": [0, 2], "u64": [1]}      # grouped by key type, arrival order kept
    assert [r.rid for r in adm.waiting] == [3]       # not arrived yet
    for _, _, res in out:
        adm.release(res)
    assert arena.used == 0


def test_admission_waits_for_memory():
    # the budget holds one big request at a time
    big = 20_000
    need = sum(serve.batch_bytes("u32", [big], _ws).values())
    arena = serve.Arena(int(need * 1.5))
    adm = serve.Admission(arena, _ws)
    a, b = serve.Request(0, "u32", big, 0.0), serve.Request(1, "u32", big, 0.0)
    adm.arrive(a)
    adm.arrive(b)
    first = adm.take(now=0.0)
    assert [r.rid for _, rs, _ in first for r in rs] == [0]
    assert adm.take(now=0.0) == []                   # b waits for memory
    adm.release(first[0][2])
    second = adm.take(now=0.0)
    assert [r.rid for _, rs, _ in second for r in rs] == [1]


def test_request_stream_shape():
    reqs = serve.make_requests(10_000, seed=11, rate_per_s=1000.0)
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 1 << 14 and sizes.max() <= 1 << 26
    assert abs(np.log2(sizes).mean() - 20.0) < 0.2          # log-uniform on [14, 26]
    kinds = [r.key_type for r in reqs]
    assert abs(kinds.count("u32") / 1e4 - 0.60) < 0.02
    assert abs(kinds.count("u64") / 1e4 - 0.25) < 0.02
    assert abs(kinds.count("f32") / 1e4 - 0.15) < 0.02
    gaps = np.diff([r.arrival for r in reqs])
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1e-3) < 1e-4  # Poisson at 1000/s
