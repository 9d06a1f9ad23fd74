"""Host logic of bench.py that needs no GPU: the order of the end-to-end
pipeline's pushes, runs and read-backs over two alternating batches."""
import concurrent.futures
import threading

import pytest

import bench


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_pipelined_steps_stage_run_drain_each_step_once_in_order(n):
    lock = threading.Lock()
    log = []
    bufs = ({"name": "a"}, {"name": "b"})
    counter = {"staged": 0}

    def stage(x):
        with lock:
            assert x.get("state") in (None, "drained"), x
            x["step"] = counter["staged"]
            counter["staged"] += 1
            x["state"] = "staged"
            log.append(("stage", x["step"]))

    def run(x):
        with lock:
            assert x["state"] == "staged", x
            x["state"] = "ran"
            log.append(("run", x["step"]))

    def drain(x):
        with lock:
            assert x["state"] == "ran", x
            x["state"] = "drained"
            log.append(("drain", x["step"]))

    with concurrent.futures.ThreadPoolExecutor(max_workers=1) as pool:
        bench.pipelined_steps(n, bufs, stage, run, drain, pool.submit)
    for what in ("stage", "run", "drain"):
        assert sorted(k for w, k in log if w == what) == list(range(n)), (what, log)
    pos = {e: i for i, e in enumerate(log)}
    for k in range(n):
        assert pos[("stage", k)] < pos[("run", k)] < pos[("drain", k)]
        if k + 1 < n:   # runs are in step order
            assert pos[("run", k)] < pos[("run", k + 1)]
    # step k runs on buffer k % 2
    assert all(b["state"] == "drained" for b in bufs[:min(n, 2)])


def test_pipelined_steps_overlaps_the_side_work_with_the_run():
    """Step k+1's staging runs while step k's run is in progress: each run
    (but the last) waits for the next step's staging, which only a helper
    working beside it can provide."""
    n = 4
    staged = [threading.Event() for _ in range(n)]
    count = {"stage": 0, "run": 0}
    seen = []

    def stage(x):
        staged[count["stage"]].set()
        count["stage"] += 1

    def run(x):
        k = count["run"]
        count["run"] += 1
        if k + 1 < n:
            seen.append(staged[k + 1].wait(timeout=5.0))

    with concurrent.futures.ThreadPoolExecutor(max_workers=1) as pool:
        bench.pipelined_steps(n, ("a", "b"), stage, run, lambda x: None, pool.submit)
    assert seen == [True] * (n - 1)
