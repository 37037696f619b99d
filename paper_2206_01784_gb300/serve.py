"""Continuous-batching sort service on one GPU.

Requests (key type, number of keys, arrival time) arrive over time. The
server admits them, in arrival order, against a fixed device-memory budget
that must hold each admitted request's input, output and its share of the
sort's workspace; requests that do not fit wait until completed work frees
memory. Whenever fewer than ``max_inflight`` batches are on the device, the
requests that arrived meanwhile are admitted, grouped by key type, and each
group becomes ONE segmented sort (os_sort_batch): the segments are the
requests; requests that arrive while the limit is reached coalesce into the
next batch. Measured on GB300 (10 000 requests, bench workload): when the
sorts bound the service (request data already in device memory), a limit of
two batches per compute stream lowers p50 and p99 at every load (0.9x
capacity: p50 5.6 vs 17.2 ms, p99 33 vs 58 ms, 2.5 requests per batch); when
each request's upload from host memory bounds it, batching saves no copy
bytes and a limit only delays uploads (p99 55 vs 41 ms at 0.7x, capacity
19.4 vs 20.8 GKeys/s), so there is none by default.
Host-to-device copies run on a copy stream, sorts on a small pool of compute
streams, so a batch's upload, other batches' sorts and completions overlap.
With ``device_resident=True`` the request data is staged in device memory
once beforehand and batches gather it with device-to-device copies: the
capacity measured that way is the sort's, not the host link's. Results stay on the device (a request's sorted keys
and values live in its batch's output buffers until the request is released).
Latency is measured from a request's arrival to its batch's completion on the
device (CUDA events), and reported as p50/p99 beside throughput.

Batching never changes a result: os_sort_batch sorts every segment on its own,
so each request gets exactly the bytes a standalone sort would give it
(tests/test_gpu_serve.py checks this request by request).

The memory bookkeeping (``Arena``) and the admission/batching policy
(``Admission``) are plain host logic and are tested without a GPU.
"""
from __future__ import annotations

import bisect
import dataclasses
import gc
import math
import time

import numpy as np

from . import onesweep as osw
from . import workload

KEY_BYTES = {"u32": 4, "u64": 8, "f32": 4, "f64": 8}
ALIGN = 256


def _round(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


@dataclasses.dataclass
class Request:
    rid: int
    key_type: str
    n: int
    arrival: float            # seconds after the start of the run
    data_offset: int = 0      # element offset of its keys in the host data pool
    admitted: float = math.nan
    done: float = math.nan    # seconds after the start (device completion)
    batch: int = -1           # batch id
    segment: int = -1         # its segment within the batch
    priority: float = math.nan  # admission priority (lower first), set once when first seen


class Arena:
    """First-fit allocator over one fixed device buffer (the memory budget).

    Offsets are bytes from the buffer's start; blocks are 256-byte aligned.
    Freed neighbours coalesce."""

    def __init__(self, capacity: int):
        self.capacity = capacity // ALIGN * ALIGN
        self.free_list = [(0, self.capacity)]  # sorted (offset, size)
        self.used = 0

    def alloc(self, nbytes: int):
        size = _round(max(nbytes, 1))
        for i, (off, sz) in enumerate(self.free_list):
            if sz >= size:
                if sz == size:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + size, sz - size)
                self.used += size
                return off
        return None

    def free(self, off: int, nbytes: int) -> None:
        size = _round(max(nbytes, 1))
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, size))
        self.used -= size
        # coalesce with the right neighbour, then the left one
        if i + 1 < len(self.free_list) and off + size == self.free_list[i + 1][0]:
            self.free_list[i] = (off, size + self.free_list[i + 1][1])
            self.free_list.pop(i + 1)
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == self.free_list[i][0]:
            self.free_list[i - 1] = (self.free_list[i - 1][0], self.free_list[i - 1][1] + self.free_list[i][1])
            self.free_list.pop(i)


def batch_bytes(key_type: str, sizes: list[int], workspace_bytes) -> dict:
    """Device bytes of one batch: keys and values in and out, the segment
    offsets, plus workspace."""
    n = sum(sizes)
    kb = KEY_BYTES[key_type]
    return {"keys_in": n * kb, "vals_in": n * 4, "keys_out": n * kb, "vals_out": n * 4,
            "seg": 8 * (len(sizes) + 1), "ws": workspace_bytes(key_type, n, len(sizes))}


class Admission:
    """Arrival-order admission against an Arena, grouped by key type.

    ``take(now)`` returns the batches to launch: {key_type: [requests]}, each
    group already holding its reservation in the arena (``reservations``)."""

    def __init__(self, arena: Arena, workspace_bytes, max_batch_keys: int = 1 << 30, order=None):
        """order: None for first-come-first-served, or a callable mapping
        requests to {id(request): priority} (lower first), as
        learned.CostModel.priority does with predicted device times. It is
        called once per request, with the requests first seen at a tick."""
        self.arena = arena
        self.workspace_bytes = workspace_bytes
        self.max_batch_keys = max_batch_keys
        self.order = order
        self.waiting: list[Request] = []

    def arrive(self, req: Request) -> None:
        self.waiting.append(req)

    def _reserve(self, key_type: str, reqs: list[Request]):
        parts = batch_bytes(key_type, [r.n for r in reqs], self.workspace_bytes)
        got = {}
        for name, nbytes in parts.items():
            off = self.arena.alloc(nbytes)
            if off is None:
                for k, (o, b) in got.items():
                    self.arena.free(o, b)
                return None
            got[name] = (off, nbytes)
        return got

    def take(self, now: float):
        """Admit waiting requests (FIFO; a request that does not fit blocks the
        ones behind it) and return [(key_type, requests, reservation)]."""
        groups: dict[str, list[Request]] = {}
        order: list[str] = []
        admitted = 0
        arrived = [r for r in self.waiting if r.arrival <= now]
        if self.order is not None and arrived:
            # a request's priority is computed once, when it is first seen (the
            # loop is latency-bound host code: nothing per request per tick)
            new = [r for r in arrived if math.isnan(r.priority)]
            if new:
                prio = self.order(new)
                for r in new:
                    r.priority = float(prio[id(r)])
            arrived.sort(key=lambda r: (r.priority, r.arrival, r.rid))
        keys_in_group: dict[str, int] = {}
        for r in arrived:
            g = groups.setdefault(r.key_type, [])
            if not g:
                order.append(r.key_type)
            if g and keys_in_group.get(r.key_type, 0) + r.n > self.max_batch_keys:
                break  # a request alone may exceed the cap; otherwise the group is full
            g.append(r)
            keys_in_group[r.key_type] = keys_in_group.get(r.key_type, 0) + r.n
            admitted += 1
        out = []
        kept = 0
        for kt in order:
            reqs = groups[kt]
            res = self._reserve(kt, reqs)
            while res is None and reqs:
                reqs = reqs[:-1]  # shrink the group until it fits
                res = self._reserve(kt, reqs) if reqs else None
            if res is None:
                continue
            for r in reqs:
                r.admitted = now
            out.append((kt, reqs, res))
            kept += len(reqs)
        taken = {id(r) for _, reqs, _ in out for r in reqs}
        self.waiting = [r for r in self.waiting if id(r) not in taken]
        return out

    def release(self, reservation) -> None:
        for off, nbytes in reservation.values():
            self.arena.free(off, nbytes)


def make_requests(count: int, seed: int, rate_per_s: float, lo_log2: int = 14, hi_log2: int = 26,
                  mix=(("u32", 0.60), ("u64", 0.25), ("f32", 0.15))) -> list[Request]:
    """Poisson arrivals at ``rate_per_s``, sizes log-uniform in [2^lo, 2^hi],
    key types drawn with the given weights (seeded, counter-based draws)."""
    u_gap = workload.uniform01(count, seed, stream=21)
    u_size = workload.uniform01(count, seed, stream=22)
    u_type = workload.uniform01(count, seed, stream=23)
    gaps = -np.log1p(-u_gap) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp2(lo_log2 + u_size * (hi_log2 - lo_log2))).astype(np.int64)
    cum = np.cumsum([w for _, w in mix])
    cum = cum / cum[-1]
    reqs = []
    for i in range(count):
        kt = mix[int(np.searchsorted(cum, u_type[i], side="right"))][0] if u_type[i] < 1.0 else mix[-1][0]
        reqs.append(Request(rid=i, key_type=kt, n=int(sizes[i]), arrival=float(arrivals[i])))
    return reqs


class Server:
    """The GPU side: owns the arena buffer, the streams and the host data pool."""

    def __init__(self, budget_bytes: int, device=None, pool_words: int = 1 << 27, compute_streams: int = 2,
                 seed: int = 11, keep_results: bool = False, small_batch_keys: int = 0,
                 device_resident: bool = False):
        """compute_streams: streams the batches rotate over. small_batch_keys >
        0 gives batches of fewer keys a higher-priority stream of their own:
        measured on the 10 000-request stream, that lowers p50 (2.8 vs 3.4 ms
        at 0.7x load) but raises p99 (21 vs 13 ms; long sorts wait behind the
        short ones, and at 0.9x their memory then holds up admission), so it
        is off by default."""
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.arena = Arena(budget_bytes)
        self.buf = torch.empty(self.arena.capacity, dtype=torch.uint8, device=self.device)
        self.base = self.buf.data_ptr()
        # host data pool (pinned): random 32-bit words; a request reads a window of it
        words = workload.u32_and(pool_words, seed, 1)
        self.pool = torch.from_numpy(words.view(np.int32)).pin_memory()
        self.iota = torch.from_numpy(workload.iota_u32(1 << 26).view(np.int32)).pin_memory()
        self.device_resident = device_resident
        if device_resident:  # staged once; batches then copy device to device
            self.dpool = self.pool.to(self.device)
            self.diota = self.iota.to(self.device)
        # page-locked staging ring for the batches' segment offsets, so the
        # loop allocates no host or device memory per batch
        self.seg_host = torch.empty(1 << 20, dtype=torch.int64).pin_memory()
        self.seg_host_np = self.seg_host.numpy()
        self.seg_pos = 0
        self.copy_stream = torch.cuda.Stream(self.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(compute_streams)]
        self.small_batch_keys = small_batch_keys
        # the short sorts' stream has the higher priority: their blocks are
        # scheduled as soon as SMs free up, ahead of a long sort's remaining ones
        self.small_stream = torch.cuda.Stream(self.device, priority=-1) if small_batch_keys > 0 else None
        self.keep_results = keep_results
        self.results = {}

    def _workspace_bytes(self, key_type, n, segs):
        b = osw.os_sort_batch_workspace_bytes(osw.KEY_TYPES[key_type], n, segs, 4, 0, 8 * KEY_BYTES[key_type])
        if b == 0:
            raise osw.OnesweepError(osw.OS_ERR_INVALID_ARG, "os_sort_batch_workspace_bytes")
        return b

    def _upload(self, key_type, reqs, res):
        """Copies every request's keys and values into the batch's input
        buffers (copy stream). Returns the segment offsets (a view of the
        batch's reservation) and the event that completes the upload."""
        torch = self.torch
        kb = KEY_BYTES[key_type]
        words_per_key = kb // 4
        pool_len = self.pool.numel()
        pool = self.dpool if self.device_resident else self.pool
        iota = self.diota if self.device_resident else self.iota
        koff = res["keys_in"][0]
        voff = res["vals_in"][0]
        offs = [0]
        with torch.cuda.stream(self.copy_stream):
            dst_k = self.buf[koff: koff + res["keys_in"][1]].view(torch.int32)
            dst_v = self.buf[voff: voff + res["vals_in"][1]].view(torch.int32)
            pos = 0
            for r in reqs:
                w = r.n * words_per_key
                start = r.data_offset % max(1, pool_len - w) if pool_len > w else 0
                src = pool[start: start + w]
                dst_k[pos * words_per_key: pos * words_per_key + w].copy_(src, non_blocking=True)
                dst_v[pos: pos + r.n].copy_(iota[: r.n], non_blocking=True)
                pos += r.n
                offs.append(pos)
            m = len(offs)
            if self.seg_pos + m > self.seg_host_np.size:
                # wrap: the staged offsets of earlier batches must have been copied
                self.copy_stream.synchronize()
                self.seg_pos = 0
            self.seg_host_np[self.seg_pos: self.seg_pos + m] = offs
            soff = res["seg"][0]
            seg = self.buf[soff: soff + 8 * m].view(torch.int64)
            seg.copy_(self.seg_host[self.seg_pos: self.seg_pos + m], non_blocking=True)
            self.seg_pos += m
        ev = torch.cuda.Event()
        ev.record(self.copy_stream)
        return seg, ev

    def run(self, requests: list[Request], tick_s: float = 0.0005, realtime: bool = True, order=None,
            max_batch_keys: int = 1 << 30, max_inflight: int | None = None) -> dict:
        """Serves the requests; returns latency and throughput statistics.
        max_inflight: batches on the device at once before new arrivals wait
        to be coalesced (default: two per compute stream for device-resident
        data, no limit when uploads from host memory bound the service)."""
        torch = self.torch
        # the loop is latency-bound host code: collect garbage now, not in the
        # middle of the run (a full collection of a previous run's objects
        # stalls every request behind it)
        gc_was_enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            if max_inflight is None:
                max_inflight = 2 * len(self.streams) if self.device_resident else 1 << 30
            return self._run(requests, tick_s, realtime, order, max_batch_keys, max_inflight)
        finally:
            if gc_was_enabled:
                gc.enable()

    def _run(self, requests, tick_s, realtime, order, max_batch_keys, max_inflight) -> dict:
        torch = self.torch
        adm = Admission(self.arena, self._workspace_bytes, max_batch_keys=max_batch_keys, order=order)
        pending = sorted(requests, key=lambda r: r.arrival)
        for i, r in enumerate(pending):
            r.data_offset = (r.rid * 7919 * 64) % max(1, self.pool.numel())
        inflight = []  # (done_event, reqs, reservation, batch_id)
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record(torch.cuda.current_stream())
        t0 = time.perf_counter()
        nxt = 0
        batch_id = 0
        rr = 0
        stats = {"batches": 0, "keys": 0}
        while nxt < len(pending) or adm.waiting or inflight:
            now = time.perf_counter() - t0 if realtime else (pending[nxt].arrival if nxt < len(pending) else 1e30)
            while nxt < len(pending) and pending[nxt].arrival <= now:
                adm.arrive(pending[nxt])
                nxt += 1
            # completions free memory
            still = []
            for ev, reqs, res, bid, ev_start in inflight:
                if ev.query():
                    t_done = t0_event.elapsed_time(ev) / 1e3
                    for r in reqs:
                        r.done = t_done
                    if not self.keep_results:
                        adm.release(res)
                else:
                    still.append((ev, reqs, res, bid, ev_start))
            inflight = still
            # a new batch only while a slot is free: arrivals meanwhile coalesce
            launched = adm.take(now) if len(inflight) < max_inflight else []
            if not launched and not inflight and adm.waiting and adm.waiting[0].arrival <= now:
                raise RuntimeError(f"request {adm.waiting[0].rid} ({adm.waiting[0].n} keys) does not fit the budget")
            for kt, reqs, res in launched:
                for j, r in enumerate(reqs):
                    r.batch, r.segment = batch_id, j
                seg, up_ev = self._upload(kt, reqs, res)
                n = sum(r.n for r in reqs)
                if self.small_stream is not None and n < self.small_batch_keys:
                    s = self.small_stream
                else:
                    s = self.streams[rr % len(self.streams)]
                    rr += 1
                s.wait_event(up_ev)
                kt_id = osw.KEY_TYPES[kt]
                ptr = lambda name: self.base + res[name][0]  # noqa: E731
                ev_start = torch.cuda.Event(enable_timing=True)
                ev_start.record(s)
                rc = osw.os_sort_batch(kt_id, ptr("keys_in"), ptr("keys_out"), ptr("vals_in"), ptr("vals_out"),
                                       seg.data_ptr(), len(reqs), n, 0, 8 * KEY_BYTES[kt], ptr("ws"),
                                       res["ws"][1], s.cuda_stream)
                if rc != osw.OS_OK:
                    raise osw.OnesweepError(rc, "os_sort_batch")
                done = torch.cuda.Event(enable_timing=True)
                done.record(s)
                seg.record_stream(s)
                inflight.append((done, reqs, res, batch_id, ev_start))
                if self.keep_results:
                    self.results[batch_id] = (kt, reqs, res)
                stats["batches"] += 1
                stats["keys"] += n
                batch_id += 1
            if realtime and nxt < len(pending) and not inflight and not adm.waiting:
                time.sleep(max(0.0, min(tick_s, pending[nxt].arrival - (time.perf_counter() - t0))))
            elif realtime:
                time.sleep(tick_s / 10)
        torch.cuda.synchronize()
        lat = np.array([r.done - r.arrival for r in requests])
        span = max(r.done for r in requests) - min(r.arrival for r in requests)
        # where the slowest 1 % spent their time: waiting for admission
        # (memory, or the requests ahead of them) or admitted and in service
        # (upload, queueing on a compute stream, the sort)
        slow = np.argsort(lat)[-max(1, len(requests) // 100):]
        wait = np.array([requests[i].admitted - requests[i].arrival for i in slow])
        serv = np.array([requests[i].done - requests[i].admitted for i in slow])
        stats.update({
            "requests": len(requests),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "tail_wait_ms": float(wait.mean() * 1e3),
            "tail_service_ms": float(serv.mean() * 1e3),
            "tail_mean_keys": float(np.mean([requests[i].n for i in slow])),
            "mean_ms": float(lat.mean() * 1e3),
            "span_s": float(span),
            "gkeys_per_s": stats["keys"] / span / 1e9,
            "mean_batch_requests": len(requests) / max(1, stats["batches"]),
        })
        return stats

    def result(self, req: Request):
        """(keys, values) device views of a finished request (keep_results=True)."""
        torch = self.torch
        kt, reqs, res = self.results[req.batch]
        kb = KEY_BYTES[kt]
        start = sum(r.n for r in reqs[: req.segment])
        k = self.buf[res["keys_out"][0] + start * kb: res["keys_out"][0] + (start + req.n) * kb]
        v = self.buf[res["vals_out"][0] + start * 4: res["vals_out"][0] + (start + req.n) * 4]
        return k, v.view(torch.int32)

    def request_input(self, req: Request):
        """The host keys of a request (as uploaded)."""
        kb = KEY_BYTES[req.key_type]
        w = req.n * (kb // 4)
        pool_len = self.pool.numel()
        start = req.data_offset % max(1, pool_len - w) if pool_len > w else 0
        return self.pool[start: start + w]
