"""CPU checks of bench.py: it parses, its reference arm prints the contract's
JSON line, and its multi-rank host logic (per-rank pairs, max-over-ranks
timing) works on world_size-2 gloo ranks."""
import json
import os
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--npairs", "2", "--n", "2048"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["metric"] == bench.METRIC


def test_overlap_macs_full_range_is_nx_times_ny():
    assert bench.overlap_macs(100, 70, -99, 69) == 100 * 70
    assert bench.overlap_macs(5, 5, 0, 0) == 5
    assert bench.overlap_macs(5, 5, 4, 4) == 1


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank times its own shard; the bench reports the slowest
    got = bench.max_over_ranks(10.0 + rank, world)
    # the learned form's agreement and in-flight flag: the smallest over ranks
    agree = bench.min_over_ranks(0.999 + 0.001 * rank, world)
    flag = bench.min_over_ranks(1.0 if rank == 0 else 0.0, world)
    q.put((rank, got, bench.rank_seed(rank), agree, flag))
    dist.barrier()
    dist.destroy_process_group()


def test_multirank_host_logic_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]          # max over ranks
    assert res[0][2] != res[1][2]                       # disjoint pairs per rank
    assert [r[3] for r in res] == [0.999, 0.999]        # min over ranks
    assert [r[4] for r in res] == [0.0, 0.0]            # one rank's flag clears it for all


def test_min_over_ranks_single_rank_is_identity():
    assert bench.min_over_ranks(0.5, 1) == 0.5
    assert bench.max_over_ranks(0.5, 1) == 0.5


def test_clock_samplers_write_separate_files():
    a, b = bench.ClockSampler(0), bench.ClockSampler(0, "learned")
    assert a.path != b.path


def test_clock_summary_parses_samples(tmp_path):
    c = bench.ClockSampler(0, "unit")
    c.path = str(tmp_path / "clocks.csv")
    c.proc = object()  # as if nvidia-smi had run
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 175.42, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 2055, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070 and s["samples"] == 2
    assert s["power_w_max"] == 175.42 and s["reasons"] == ["sw_power_cap"]
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active\n")
    assert c.summary()["power_w_max"] is None
