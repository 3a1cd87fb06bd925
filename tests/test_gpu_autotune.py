"""GPU tests of the engine autotuner: it measures every exact engine, AUTO
follows its table, results stay exact whichever engine the table picks, and
the JSON cache round-trips."""
import json

import pytest
import torch

import oracle
from paper_2509_19974_gb300 import synth, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return tde.Context(0)


def test_autotune_measures_all_engines_and_picks_the_fastest(ctx):
    pts = [(4096, 256), (65536, 131071)]
    table = ctx.autotune(2, pts, reps=2)
    got = [t for t in table if t["bits"] == 2]
    assert [(t["log2_n"], t["log2_lags"]) for t in got] == [(12, 8), (16, 17)]
    for t in got:
        ns = t["ns_per_pair"]
        assert all(v is not None and v > 0 for v in ns.values()), t
        assert t["engine"] == min(ns, key=ns.get)
        assert ctx.pick_engine(2, 1 << t["log2_n"], 1 << t["log2_n"],
                               1 << t["log2_lags"]) == t["engine"]
    # the dense full-range point is a tensor-core case on this part
    assert got[1]["engine"] in ("mma", "ntt")
    # a different bit width is untouched: built-in rule
    assert ctx.pick_engine(1, 4096, 4096, 256) == tde.pick_engine(1, 4096, 4096, 256)


@pytest.mark.parametrize("engine", ["popc", "mma", "ntt"])
def test_table_routes_auto_and_stays_exact(engine):
    ctx = tde.Context(0)
    ctx.autotune_load([{"bits": 2, "log2_n": 12, "log2_lags": 12, "engine": engine,
                        "ns_per_pair": {}}])
    assert ctx.pick_engine(2, 3000, 5000, 7000) == engine
    b = synth.uneven_batch(seed=91, npairs=6, n_lo=1500, n_hi=6000, bits=2)
    xs = [torch.from_numpy(x).cuda() for x in b.x]
    ys = [torch.from_numpy(y).cuda() for y in b.y]
    lags, vals = ctx.estimate_batch(xs, ys, 2, b.lag_min, b.lag_max)
    ctx.sync()
    for i in range(len(xs)):
        lag, val = oracle.estimate(b.x[i], b.y[i], 2, int(b.lag_min[i]), int(b.lag_max[i]))
        assert (int(lags[i]), int(vals[i])) == (lag, val), (engine, i)


def test_autotune_cache_round_trip(ctx, tmp_path):
    path = str(tmp_path / "tune.json")
    pts = [(2048, 1024)]
    t1 = tde.autotune_cached(ctx, bits_list=(1,), points=pts, path=path, reps=1)
    cache = json.load(open(path))
    assert list(cache) == [tde.tune_cache_key(0)]
    # a fresh context loads the cached table without measuring again
    ctx2 = tde.Context(0)
    t2 = tde.autotune_cached(ctx2, bits_list=(1,), points=pts, path=path, reps=1)
    assert t2 == cache[tde.tune_cache_key(0)]
    assert ctx2.autotune_table() == t1
