"""One array sorted across ranks (one process per GPU) with one exchange step.

The paper sorts an array held by one device (Section 1's problem statement).
An array spread over several GPUs shards along its most significant digit
place, because the upfront histogram (Section 3, phase 1) gives each rank the
exact count of every top digit before any key moves:

  1. every rank counts the top-place digits of its shard (the histogram
     kernel) and an all-reduce sums the counts over ranks;
  2. the top place's bins are split into ``world`` contiguous ranges of about
     n / world keys each (an MSD split; a bin is never divided, so one bin
     holding most keys lands on one rank);
  3. every rank stably partitions its shard by top digit (one binning pass
     over the top place), so each destination's keys are contiguous and in
     input order, and one all-to-all moves keys (and values);
  4. every rank sorts what it received on all bits [begin, end) with the
     single-GPU sort.

Rank r holds the r-th contiguous piece of the input. Pieces arrive in source
rank order and each stays in input order, so the received keys are in input
order and the local sort's stability makes the whole sort stable: the ranks'
outputs, concatenated in rank order, are the stable sort of the array.

The collectives are torch.distributed's (NCCL between GPUs; gloo, whose
exchange goes through host memory, for the CPU tests). The local steps run
behind a backend: ``CudaBackend`` calls the library's kernels through its C
ABI and is the only one this package provides.
"""
from __future__ import annotations

from dataclasses import dataclass

RADIX_BITS = 8


def top_place(begin_bit: int, end_bit: int) -> tuple[int, int]:
    """Bits [lo, end_bit) of the most significant digit place: places start
    at begin_bit and go up in RADIX_BITS steps, the top one possibly
    narrower."""
    if end_bit <= begin_bit:
        return begin_bit, begin_bit
    places = (end_bit - begin_bit + RADIX_BITS - 1) // RADIX_BITS
    return begin_bit + RADIX_BITS * (places - 1), end_bit


def plan_split(hist: list[int], world: int) -> list[int]:
    """Bin boundaries b[0] = 0 <= b[1] <= ... <= b[world] = len(hist): rank j
    receives the keys of bins [b[j], b[j+1]). Each inner boundary is the bin
    edge whose running count is nearest to j * total / world (the lower edge
    on a tie), never left of the previous boundary. Deterministic, and the same
    on every rank given the same summed histogram."""
    if world < 1:
        raise ValueError("world must be >= 1")
    nb = len(hist)
    total = sum(int(h) for h in hist)
    cum = [0]
    for h in hist:
        cum.append(cum[-1] + int(h))
    bounds = [0]
    e = 0
    for j in range(1, world):
        target = j * total / world
        while e < nb and cum[e + 1] <= target:
            e += 1
        # edge e has cum[e] <= target < cum[e+1] (or e == nb): take e or e+1
        best = e
        if e < nb and (cum[e + 1] - target) < (target - cum[e]):
            best = e + 1
        best = max(best, bounds[-1])
        bounds.append(best)
    bounds.append(nb)
    return bounds


def send_counts(local_hist: list[int], bounds: list[int]) -> list[int]:
    """Keys this rank sends to each rank: its own counts summed over each
    rank's bin range."""
    return [sum(int(h) for h in local_hist[bounds[j]:bounds[j + 1]]) for j in range(len(bounds) - 1)]


@dataclass
class ShardPlan:
    top_lo: int               # bits [top_lo, top_hi) of the top place
    top_hi: int
    global_hist: list[int]    # summed top-place counts, in sort order of the bins
    bounds: list[int]         # bin boundaries per rank
    send: list[int]           # keys this rank sends to each rank
    recv: list[int]           # keys this rank receives from each rank


class CudaBackend:
    """The local steps on this rank's GPU through the library's C ABI."""

    def __init__(self, key_type=None, descending: bool = False):
        from . import onesweep

        self.osw = onesweep
        self.key_type = key_type
        self.descending = descending

    def top_histogram(self, keys, lo: int, hi: int) -> list[int]:
        """Counts of the top place's digits, in the order the sort places them."""
        if keys.numel() == 0:
            return [0] * (1 << (hi - lo))
        hist, _ = self.osw.digit_histograms(keys, begin_bit=lo, end_bit=hi, key_type=self.key_type,
                                            descending=self.descending)
        return [int(x) for x in hist[0, :1 << (hi - lo)].cpu().tolist()]

    def partition(self, keys, values, lo: int, hi: int):
        """Stable partition by top digit: one binning pass over bits [lo, hi)."""
        if keys.numel() == 0:
            return keys, values
        if values is None:
            return self.osw.sort_keys(keys, begin_bit=lo, end_bit=hi, key_type=self.key_type,
                                      descending=self.descending), None
        return self.osw.sort_pairs(keys, values, begin_bit=lo, end_bit=hi, key_type=self.key_type,
                                   descending=self.descending)

    def sort(self, keys, values, begin_bit: int, end_bit: int):
        if keys.numel() == 0:
            return keys, values
        if values is None:
            return self.osw.sort_keys(keys, begin_bit=begin_bit, end_bit=end_bit, key_type=self.key_type,
                                      descending=self.descending), None
        return self.osw.sort_pairs(keys, values, begin_bit=begin_bit, end_bit=end_bit, key_type=self.key_type,
                                   descending=self.descending)


def _through_host(group) -> bool:
    import torch.distributed as dist

    return dist.get_backend(group) == "gloo"


def _all_reduce_counts(counts: list[int], device, group) -> list[int]:
    import torch
    import torch.distributed as dist

    host = _through_host(group)
    t = torch.tensor(counts, dtype=torch.int64, device="cpu" if host else device)
    dist.all_reduce(t, group=group)
    return [int(x) for x in t.cpu().tolist()]


def _exchange_counts(send: list[int], device, group) -> list[int]:
    import torch
    import torch.distributed as dist

    host = _through_host(group)
    dev = "cpu" if host else device
    s = torch.tensor(send, dtype=torch.int64, device=dev)
    r = torch.empty_like(s)
    dist.all_to_all_single(r, s, group=group)
    return [int(x) for x in r.cpu().tolist()]


def _exchange(x, send: list[int], recv: list[int], group):
    """One all-to-all of a 1-D tensor: piece j (send[j] elements, in order) to
    rank j; pieces received concatenated in source rank order."""
    import torch
    import torch.distributed as dist

    host = _through_host(group) and x.device.type != "cpu"
    src = x.cpu() if host else x
    out = torch.empty(sum(recv), dtype=x.dtype, device=src.device)
    dist.all_to_all_single(out, src.contiguous(), output_split_sizes=recv, input_split_sizes=send, group=group)
    return out.to(x.device) if host else out


def plan(keys, begin_bit: int, end_bit: int, backend, group=None) -> ShardPlan:
    """Steps 1-2 and the count exchange: the split every rank agrees on."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    lo, hi = top_place(begin_bit, end_bit)
    local = backend.top_histogram(keys, lo, hi)
    glob = _all_reduce_counts(local, keys.device, group)
    bounds = plan_split(glob, world)
    send = send_counts(local, bounds)
    recv = _exchange_counts(send, keys.device, group)
    return ShardPlan(lo, hi, glob, bounds, send, recv)


def sharded_sort(keys, values=None, begin_bit: int = 0, end_bit: int | None = None, backend=None, group=None):
    """Sorts the array whose r-th piece is this rank's ``keys`` (and
    ``values``). Returns this rank's part of the sorted array (keys, values)
    and the plan; the parts in rank order are the whole sorted array. Every
    rank of ``group`` must call it."""
    if backend is None:
        backend = CudaBackend()
    if end_bit is None:
        end_bit = keys.element_size() * 8
    if values is not None and values.numel() != keys.numel():
        raise ValueError("one value per key")
    p = plan(keys, begin_bit, end_bit, backend, group)
    k, v = backend.partition(keys, values, p.top_lo, p.top_hi)
    rk = _exchange(k, p.send, p.recv, group)
    rv = None if v is None else _exchange(v, p.send, p.recv, group)
    ok, ov = backend.sort(rk, rv, begin_bit, end_bit)
    return ok, ov, p
