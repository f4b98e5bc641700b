"""The N > 1 host path of bench.py on CPU: two ranks over gloo (no GPU).

The method shards by image subset, but every run here has one GPU, so
`bench.py --gpus N` runs N independent replicas: a barrier around the timed
region, the step time as the maximum over ranks, and no data-path collective.
These tests run that host logic as two processes: rendezvous through the same
environment torchrun sets, the max-over-ranks reduction, the barrier, the
agreement to time the steps again when any rank's clocks void its number, and
the reference arm, which only rank 0 runs (the other ranks return at once).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, n, dist = bench.dist_init("gloo")
    assert (r, n) == (rank, ws) and dist is not None
    bench.barrier(dist)
    # every rank reports its own step time; the job's time is the slowest rank's
    got = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{r} {n} {got}\n")
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    assert [(int(a), int(b)) for a, b, _ in rows] == [(0, 2), (1, 2)]
    assert all(float(c) == 15.0 for _, _, c in rows)


def _reference_rank_main(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    called = []
    # rank 0 would time the oracle; here only the rank split is checked, so the
    # estimate raises to show that rank 0, and only rank 0, reaches it
    def stop(*a, **k):
        called.append(1)
        raise RuntimeError("rank 0 reached the oracle")
    bench.oracle_step_entries_estimate = stop
    args = bench.parse_args(["--impl", "reference", "--gpus", str(ws), "--steps", "1", "--warmup", "0"])
    try:
        rc = bench.run_reference(args)
        result = f"returned {rc}"
    except RuntimeError as e:
        result = str(e)
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(result + "\n")


def test_reference_arm_runs_on_rank_0_only(tmp_path):
    port = _free_port()
    mp.spawn(_reference_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert open(tmp_path / "ref0.txt").read().strip() == "rank 0 reached the oracle"
    assert open(tmp_path / "ref1.txt").read().strip() == "returned 0"


def _remeasure_rank_main(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, n, dist = bench.dist_init("gloo")
    # only rank 1's GPU throttled: both ranks must time the steps again, or the
    # rank that does would wait at the barrier alone
    why = "slowdown: hw_thermal_slowdown" if rank == 1 else ""
    first = bench.agree_remeasure(why, dist, "cpu")
    second = bench.agree_remeasure("", dist, "cpu")
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"re{rank}.txt"), "w") as f:
        f.write(f"{int(first)} {int(second)}\n")
    dist.destroy_process_group()


def test_ranks_agree_to_measure_again(tmp_path):
    port = _free_port()
    mp.spawn(_remeasure_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert [open(tmp_path / f"re{r}.txt").read().split() for r in range(2)] == [["1", "0"], ["1", "0"]]


def test_single_rank_needs_no_process_group(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    import bench
    rank, ws, dist = bench.dist_init("gloo")
    assert (rank, ws, dist) == (0, 1, None)
    assert bench.max_over_ranks(3.5, dist) == 3.5
    bench.barrier(dist)
