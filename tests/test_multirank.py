"""The multi-rank path of bench.py on host ranks (gloo, world size 2).

Windows are independent, so ranks run replicas with no data-path
collective: each rank takes its own windows, the step time is the slowest
rank's and the throughput counts every rank's units.  For the reference arm
rank 0 alone runs the oracle and prints the line; the other ranks leave
without work."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)


def _reduction_rank(rank, world, port, out_dir):
    _env(rank, world, port)
    import bench
    r, w, local, pg = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank) and pg.get_backend() == "gloo"
    mx = bench.max_over_ranks(pg, float(rank + 1), "cpu")
    ms, rate = bench.whole_job(pg, world, 1000.0, 500.0 * (rank + 1), "cpu")
    seeds = bench.rank_window_seeds(2000, rank, 8)
    everyone = [None] * world
    pg.all_gather_object(everyone, seeds)
    bench.barrier(pg)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": mx, "ms": ms, "rate": rate, "seeds": everyone}, f)
    pg.destroy_process_group()


def _reference_rank(rank, world, port, out_dir):
    _env(rank, world, port)
    import bench
    calls = []

    def fake_sample(cw=608, ch=184):   # the signature of bench.oracle_sample
        calls.append((cw, ch))
        return 1.0e5, 2.0, f"fake sample {cw}x{ch}"

    def fake_all_cores():              # the signature of bench.oracle_all_cores
        calls.append(("all", 16))
        return 1.0e5, 2.0, 16, "fake all-cores step 1216x368"

    bench.oracle_sample = fake_sample
    bench.oracle_all_cores = fake_all_cores
    out = os.path.join(out_dir, f"ref{rank}.txt")
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "3",
                "--warmup", "2"]
    stdout = sys.stdout
    with open(out, "w") as f:
        sys.stdout = f
        try:
            rc = bench.main()
        finally:
            sys.stdout = stdout
    with open(os.path.join(out_dir, f"ref{rank}.calls.json"), "w") as f:
        json.dump({"rc": rc, "calls": calls}, f)


@pytest.mark.timeout(300)
def test_replicas_reduce_to_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_reduction_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["max"] == 2.0
        assert r["ms"] == 1000.0                          # the slower rank's time
        assert r["rate"] == pytest.approx(1000.0 * world / 1.0)   # units of all ranks / that time
    seeds = res[0]["seeds"]
    assert seeds == res[1]["seeds"]
    flat = [s for rank_seeds in seeds for s in rank_seeds]
    assert len(set(flat)) == len(flat)                    # no window is run twice


@pytest.mark.timeout(300)
def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    world = 2
    mp.spawn(_reference_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = json.load(open(tmp_path / "ref0.calls.json"))
    r1 = json.load(open(tmp_path / "ref1.calls.json"))
    assert r0["rc"] == 0 and r1["rc"] == 0
    assert len(r0["calls"]) == 2 + 3 and r1["calls"] == []    # warm-up + timed steps, rank 0 only
    assert r0["calls"][:2] == [[304, 92]] * 2                 # warm-up on the small crop
    assert r0["calls"][2:] == [["all", 16]] * 3               # the timed steps on every core
    assert open(tmp_path / "ref1.txt").read() == ""
    lines = open(tmp_path / "ref0.txt").read().strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 2
    assert line["value"] == 1.0e5 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the contract's keys, the same metric, unit and workload as our arm's line
    import bench
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["vs_baseline"] is None and line["data"] == "synthetic" and line["n_gpus"] == 1
    cfg = dict(line["config"])
    assert cfg.pop("reference_step") == "fake all-cores step 1216x368"
    assert cfg == bench.workload_config(8, 1)
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["value"] == line["value"] and cb["cores"] == 16 and cb["host"]["nproc"] >= 1
    assert "1216x368" in cb["sample"] and line["ms_per_step"] > 0
