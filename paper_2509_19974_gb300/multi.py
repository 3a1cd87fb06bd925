"""The estimator over several ranks (one process per GPU).

Pairs are independent, so a batch of uneven pairs is split by cost with the
longest-processing-time rule (``lpt_partition``): each rank runs its share with
no exchange, and only the lags are gathered.

One long template search (a short y inside a long x) is split by lag instead.
``lag_shards`` gives every rank a contiguous range of lags; the rank correlates
its range through the library (every rank holds both signals and quantizes
them whole, because the rank quantizer's thresholds are order statistics of
the whole signal) and takes the tie-ruled argmax of its range. The ranks then
agree on the global answer (``reduce_argmax``) with one max-reduce of the
values and one min-reduce of the lags' tie ranks among the ranks that hold
the maximum. The order is the single-GPU argmax's (Algorithm 1's argmax step,
with ties to the smallest |tau|, then the smallest tau), so the sharded answer
equals the unsharded one.
"""
from __future__ import annotations

import heapq

import torch
import torch.distributed as dist

_NONE = -(1 << 62)  # value of a rank with an empty lag range
_WORST = 1 << 62    # tie rank of a rank without the maximum


def lpt_partition(costs, world: int) -> list[list[int]]:
    """Pair indices per rank: pairs in decreasing cost, each to the rank with
    the least load so far (lower rank on equal load); indices sorted per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(o) for o in out]


def lag_shards(lag_min: int, lag_max: int, world: int) -> list[tuple[int, int]]:
    """Contiguous lag ranges (lo, hi), one per rank, sizes differing by at most
    one; a range with hi < lo is empty."""
    if world < 1 or lag_max < lag_min:
        raise ValueError("need world >= 1 and lag_min <= lag_max")
    count = lag_max - lag_min + 1
    return [(lag_min + count * r // world, lag_min + count * (r + 1) // world - 1)
            for r in range(world)]


def tie_rank(lag: int) -> int:
    """Order of equal maxima: smaller |lag| first, then the negative lag."""
    return 2 * abs(lag) + (1 if lag > 0 else 0)


def rank_to_lag(rk: int) -> int:
    a = rk // 2
    return a if rk & 1 else -a


def combine_argmax(locals_) -> tuple[int, int]:
    """reduce_argmax's answer from all ranks' (lag, val) at once (host side)."""
    held = [(l, v) for l, v in locals_ if v is not None]
    if not held:
        raise ValueError("no rank holds a lag")
    vmax = max(v for _, v in held)
    return min((l for l, v in held if v == vmax), key=tie_rank), vmax


def reduce_argmax(lag, val, group=None, device="cpu") -> tuple[int, int]:
    """The tie-ruled argmax over all ranks from each rank's local one (lag,
    val), or (None, None) for a rank with no lags.  Returns (lag, value) on
    every rank."""
    v = torch.tensor([_NONE if val is None else int(val)], dtype=torch.int64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX, group=group)
    vmax = int(v.item())
    if vmax == _NONE:
        raise ValueError("no rank holds a lag")
    rk = torch.tensor([tie_rank(int(lag)) if val is not None and int(val) == vmax else _WORST],
                      dtype=torch.int64, device=device)
    dist.all_reduce(rk, op=dist.ReduceOp.MIN, group=group)
    return rank_to_lag(int(rk.item())), vmax


def shard_argmax(ctx, qx: torch.Tensor, qy: torch.Tensor, bits: int, lo: int, hi: int,
                 engine: str = "auto"):
    """One rank's share: the tie-ruled argmax of the quantized pair over the
    lags [lo, hi] (int64 correlations), or (None, None) when hi < lo."""
    if hi < lo:
        return None, None
    c = ctx.xcorr_int(qx, qy, bits, lo, hi, engine=engine, dtype=torch.int64)
    lt, vt = ctx.argmax(c, lo)
    ctx.sync()
    return int(lt.item()), int(vt.item())


def template_search(ctx, x: torch.Tensor, y: torch.Tensor, bits: int, lag_min: int, lag_max: int,
                    group=None, engine: str = "auto") -> tuple[int, int]:
    """Algorithm 1 for one pair over the lags [lag_min, lag_max], split by lag
    over the ranks of ``group`` (or run whole without torch.distributed). x, y:
    FP32 on this rank's GPU. Correlations are int64. Returns (lag, value)."""
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    lo, hi = lag_shards(lag_min, lag_max, world)[rank]
    qx, qy = ctx.quantize(x, bits), ctx.quantize(y, bits)
    lag, val = shard_argmax(ctx, qx, qy, bits, lo, hi, engine)
    if world == 1:
        return lag, val
    device = x.device if dist.get_backend(group) == "nccl" else "cpu"
    return reduce_argmax(lag, val, group, device)
