"""Host logic of the multi-rank forms (no GPU): cost partition of uneven
pairs, lag shards of one long search, and the cross-rank tie-ruled argmax on
world_size-2 gloo ranks, checked against the oracle's unsharded argmax."""
import os
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_2509_19974_gb300 import multi  # noqa: E402


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(3)
    costs = [int(c) for c in rng.integers(1, 1000, 97)]
    for world in (1, 2, 3, 8):
        parts = multi.lpt_partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # the LPT bound: no rank exceeds the mean load by more than one pair
        assert max(loads) <= sum(costs) / world + max(costs)
    assert multi.lpt_partition([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]


def test_lag_shards_are_contiguous_and_exact():
    for lo, hi, world in ((-10, 10, 3), (0, 0, 4), (-65535, 65535, 8), (5, 6, 2)):
        sh = multi.lag_shards(lo, hi, world)
        assert len(sh) == world and sh[0][0] == lo and sh[-1][1] == hi
        for (a, b), (c, _) in zip(sh, sh[1:]):
            assert c == b + 1
        sizes = [b - a + 1 for a, b in sh]
        assert max(sizes) - min(sizes) <= 1 and sum(sizes) == hi - lo + 1


def test_tie_rank_order():
    lags = [3, -3, 0, 1, -1, 7, -7]
    assert sorted(lags, key=multi.tie_rank) == [0, -1, 1, -3, 3, -7, 7]
    for lag in range(-20, 21):
        assert multi.rank_to_lag(multi.tie_rank(lag)) == lag


def _rank(rank, world, port, cases, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    for c, lo in cases:
        hi = lo + len(c) - 1
        a, b = multi.lag_shards(lo, hi, world)[rank]
        local = oracle.argmax(c[a - lo: b - lo + 1], a) if b >= a else (None, None)
        out.append(multi.reduce_argmax(local[0], local[1]))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_argmax_equals_unsharded_gloo():
    rng = np.random.default_rng(11)
    cases = []
    # exact correlations of quantized random pairs
    for n in (7, 33, 64):
        qx = rng.integers(-1, 2, n).astype(np.int8)
        qy = rng.integers(-1, 2, n).astype(np.int8)
        cases.append((oracle.xcorr(qx, qy, -(n - 1), n - 1), -(n - 1)))
    # ties that straddle the shards: equal maxima at -4 and +4 (and 5), smaller |tau| wins
    c = np.zeros(21, dtype=np.int64)
    c[[6, 14, 15]] = 9  # lags -4, 4, 5
    cases.append((c, -10))
    c = np.full(9, -3, dtype=np.int64)  # constant: lag 0 wins
    cases.append((c, -4))
    c = np.zeros(3, dtype=np.int64)
    c[[0, 2]] = 1  # lags -1 and +1 tie, on different ranks: -1
    cases.append((c, -1))
    ctx = mp.get_context("spawn")
    for world in (2, 3):
        q = ctx.Queue()
        port = 29700 + 10 * world + os.getpid() % 100
        procs = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
        for p in procs:
            p.start()
        res = [q.get(timeout=120) for _ in procs]
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
        want = [oracle.argmax(cc, lo) for cc, lo in cases]
        for _, got in res:
            assert got == want


def test_combine_argmax_matches_oracle_on_shards():
    rng = np.random.default_rng(5)
    for n in (9, 40):
        qx = rng.integers(-1, 2, n).astype(np.int8)
        qy = rng.integers(-1, 2, n).astype(np.int8)
        lo, hi = -(n - 1), n - 1
        c = oracle.xcorr(qx, qy, lo, hi)
        for world in (1, 2, 5, 2 * n - 1):
            locs = [oracle.argmax(c[a - lo: b - lo + 1], a) if b >= a else (None, None)
                    for a, b in multi.lag_shards(lo, hi, world)]
            assert multi.combine_argmax(locs) == oracle.argmax(c, lo)
